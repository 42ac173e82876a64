// Gradient of the rate surrogate without any device allocation.
//
// dmb_surrogate_grad allocates its per-batch work buffers with cudaMalloc on every call.  Some
// callers cannot do that: code that runs while a CUDA graph is being captured, code under an
// external memory manager that owns every allocation, or real-time loops where a cudaMalloc /
// cudaFree (which can synchronise the device) is not acceptable.  This variant runs the same
// kernels with its work buffers in one file-scope device array of fixed size, so the call itself
// allocates nothing.  The array lives on every GPU that loads the library until the process exits.
#include <mutex>

#include "internal.cuh"
#include "mlp.cuh"

#define NOALLOC_MAX_BATCH 4096

namespace {
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kBH = (size_t)NOALLOC_MAX_BATCH * MLP_H;
constexpr size_t kOffIdx = 0;
constexpr size_t kOffA1 = align256(kOffIdx + NOALLOC_MAX_BATCH * sizeof(int));
constexpr size_t kOffA2 = align256(kOffA1 + kBH * 2);
constexpr size_t kOffDZ3 = align256(kOffA2 + kBH * 2);
constexpr size_t kOffDZ2 = align256(kOffDZ3 + kBH * 2);
constexpr size_t kOffZ1 = align256(kOffDZ2 + kBH * 2);
constexpr size_t kOffZ2 = align256(kOffZ1 + kBH * 4);
constexpr size_t kOffZ3 = align256(kOffZ2 + kBH * 4);
constexpr size_t kOffA3 = align256(kOffZ3 + kBH * 4);
constexpr size_t kOffDZ1 = align256(kOffA3 + kBH * 4);
constexpr size_t kOffDY = align256(kOffDZ1 + kBH * 4);
constexpr size_t kOffLoss = align256(kOffDY + (size_t)NOALLOC_MAX_BATCH * 2 * 4);
constexpr size_t kOffP2 = align256(kOffLoss + MLP_TRAIN_BLOCKS * 4);
constexpr size_t kOffP3 = align256(kOffP2 + (size_t)MLP_KSLICES * MLP_H * MLP_H * 4);
constexpr size_t kBytes = align256(kOffP3 + (size_t)MLP_KSLICES * MLP_H * MLP_H * 4);   // about 16 MB
}  // namespace

// The work buffers (shared by every call on a device; they keep the last call's contents).
static __device__ __align__(256) unsigned char g_surrogate_grad_scratch[kBytes];

__global__ void k_noalloc_iota(int *idx, int B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < B) idx[t] = t;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

// Device address of the array for the current device, looked up once per device.  Host code
// must not hand the symbol itself to a kernel: on the host it names a stand-in, not device memory.
cudaError_t scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_surrogate_grad_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" dmb_status dmb_surrogate_grad_noalloc(dmb_ctx *ctx, const float *X, const float *Y, int32_t B, float *grad,
                                                  double *loss) {
  if (!ctx) return dmb_internal_fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  MlpDev d;
  cudaStream_t s;
  if (!dmb_internal_surrogate(ctx, &d, &s)) return dmb_internal_fail(ctx, DMB_ERR_STATE, "no surrogate loaded");
  if (B < 1 || B > NOALLOC_MAX_BATCH)
    return dmb_internal_fail(ctx, DMB_ERR_ARG,
                             "dmb_surrogate_grad_noalloc: batch size must be in [1, 4096] (its fixed work array)");
  if (!X || !Y || !grad) return dmb_internal_fail(ctx, DMB_ERR_ARG, "NULL array");
  // the array is per device: the one to use is that of the device the context's stream is on
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != dmb_internal_device(ctx)) {
    cudaGetLastError();
    return dmb_internal_fail(ctx, DMB_ERR_STATE,
                             "dmb_surrogate_grad_noalloc: the current CUDA device is not the context's device");
  }
  unsigned char *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return dmb_internal_fail(ctx, DMB_ERR_CUDA, cudaGetErrorString(e));
  // every buffer below is written before it is read within the call, so nothing is cleared
  MlpWork w;
  int *idx = reinterpret_cast<int *>(base + kOffIdx);
  w.A1 = reinterpret_cast<__nv_bfloat16 *>(base + kOffA1);
  w.A2 = reinterpret_cast<__nv_bfloat16 *>(base + kOffA2);
  w.dZ3 = reinterpret_cast<__nv_bfloat16 *>(base + kOffDZ3);
  w.dZ2 = reinterpret_cast<__nv_bfloat16 *>(base + kOffDZ2);
  w.Z1 = reinterpret_cast<float *>(base + kOffZ1);
  w.Z2 = reinterpret_cast<float *>(base + kOffZ2);
  w.Z3 = reinterpret_cast<float *>(base + kOffZ3);
  w.A3 = reinterpret_cast<float *>(base + kOffA3);
  w.dZ1 = reinterpret_cast<float *>(base + kOffDZ1);
  w.dY = reinterpret_cast<float *>(base + kOffDY);
  w.loss = reinterpret_cast<float *>(base + kOffLoss);
  w.part2 = reinterpret_cast<float *>(base + kOffP2);
  w.part3 = reinterpret_cast<float *>(base + kOffP3);
  w.grad = grad;
  k_noalloc_iota<<<(B + 255) / 256, 256, 0, s>>>(idx, B);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = mlp_grad(d, X, Y, idx, B, w, s);
  float lh[MLP_TRAIN_BLOCKS];
  if (e == cudaSuccess && loss) {
    e = cudaMemcpyAsync(lh, w.loss, sizeof(lh), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      double t = 0.0;
      for (int k = 0; k < MLP_TRAIN_BLOCKS; ++k) t += lh[k];
      *loss = t / (double)B;
    }
  }
  if (e != cudaSuccess) return dmb_internal_fail(ctx, DMB_ERR_CUDA, cudaGetErrorString(e));
  return DMB_OK;
}
