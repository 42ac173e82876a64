// Throughput probe of the arithmetic pipes the pair kernels use: float32 FMA, float64 FMA,
// the special-function unit (ex2, tanh), int32 multiply-add, 32-bit multiply-high (Philox)
// and the warp-level bf16 tensor instruction (mma.sync m16n8k16) of the surrogate.
// Independent chains per thread; every thread writes one word so nothing is dead code.
// Built and run by paper_2603_24688_gb300/peaks.py; not part of libdmb.so.
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
__global__ void k_ffma(float* out, float a, float b) {
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i=0;i<ITERS;i++){ x0=fmaf(x0,a,b);x1=fmaf(x1,a,b);x2=fmaf(x2,a,b);x3=fmaf(x3,a,b);
    x4=fmaf(x4,a,b);x5=fmaf(x5,a,b);x6=fmaf(x6,a,b);x7=fmaf(x7,a,b);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void k_dfma(double* out, double a, double b) {
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i=0;i<ITERS/8;i++){ x0=fma(x0,a,b);x1=fma(x1,a,b);x2=fma(x2,a,b);x3=fma(x3,a,b);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
__global__ void k_mufu(float* out, float a) {
  float x0=threadIdx.x*1e-3f, x1=x0+1e-3f, x2=x0+2e-3f, x3=x0+3e-3f;
  for (int i=0;i<ITERS/4;i++){ x0=exp2f(x0)*a; x1=exp2f(x1)*a; x2=exp2f(x2)*a; x3=exp2f(x3)*a; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
__global__ void k_imad(unsigned* out, unsigned a, unsigned b) {
  unsigned x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i=0;i<ITERS;i++){ x0=x0*a+b;x1=x1*a+b;x2=x2*a+b;x3=x3*a+b;x4=x4*a+b;x5=x5*a+b;x6=x6*a+b;x7=x7*a+b;}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0^x1^x2^x3^x4^x5^x6^x7;
}
__global__ void k_mulhi(unsigned* out, unsigned a) {
  unsigned x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i=0;i<ITERS;i++){ x0=__umulhi(x0,a)^x0;x1=__umulhi(x1,a)^x1;x2=__umulhi(x2,a)^x2;x3=__umulhi(x3,a)^x3;}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0^x1^x2^x3;
}
__global__ void k_tanh(float* out, float a) {
  float x0=threadIdx.x*1e-3f, x1=x0+1e-3f, x2=x0+2e-3f, x3=x0+3e-3f;
  for (int i=0;i<ITERS/4;i++){
    asm volatile("tanh.approx.f32 %0, %0;" : "+f"(x0)); asm volatile("tanh.approx.f32 %0, %0;" : "+f"(x1));
    asm volatile("tanh.approx.f32 %0, %0;" : "+f"(x2)); asm volatile("tanh.approx.f32 %0, %0;" : "+f"(x3));
    x0*=a; x1*=a; x2*=a; x3*=a; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
__global__ void k_tanh2(float* out, unsigned a) {
  unsigned x0=threadIdx.x*0x00010001u, x1=x0^0x3c003c00u, x2=x0^0x3d003d00u, x3=x0^0x3e003e00u;
  for (int i=0;i<ITERS/4;i++){
    asm volatile("tanh.approx.bf16x2 %0, %0;" : "+r"(x0)); asm volatile("tanh.approx.bf16x2 %0, %0;" : "+r"(x1));
    asm volatile("tanh.approx.bf16x2 %0, %0;" : "+r"(x2)); asm volatile("tanh.approx.bf16x2 %0, %0;" : "+r"(x3));
    x0^=a; x1^=a; x2^=a; x3^=a; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=(float)(x0^x1^x2^x3);
}
__global__ void k_tanhh2(float* out, unsigned a) {
  unsigned x0=0x3c003c00u^threadIdx.x, x1=x0^0x00010001u, x2=x0^0x00020002u, x3=x0^0x00030003u;
  for (int i=0;i<ITERS/4;i++){
    asm volatile("tanh.approx.f16x2 %0, %0;" : "+r"(x0)); asm volatile("tanh.approx.f16x2 %0, %0;" : "+r"(x1));
    asm volatile("tanh.approx.f16x2 %0, %0;" : "+r"(x2)); asm volatile("tanh.approx.f16x2 %0, %0;" : "+r"(x3));
    x0^=a; x1^=a; x2^=a; x3^=a; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=(float)(x0^x1^x2^x3);
}
__global__ void k_ex2h2(float* out, unsigned a) {
  unsigned x0=0x3c003c00u^threadIdx.x, x1=x0^0x00010001u, x2=x0^0x00020002u, x3=x0^0x00030003u;
  for (int i=0;i<ITERS/4;i++){
    asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(x0)); asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(x1));
    asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(x2)); asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(x3));
    x0^=a; x1^=a; x2^=a; x3^=a; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=(float)(x0^x1^x2^x3);
}
// 4 independent m16n8k16 bf16 accumulator chains per warp; 4096 flops per instruction
__global__ void k_mma(float* out, unsigned a) {
  unsigned A0=a^threadIdx.x, A1=A0*3u, A2=A0*5u, A3=A0*7u, B0=A0*11u, B1=A0*13u;
  float c[4][4];
  for (int k=0;k<4;k++) for (int q=0;q<4;q++) c[k][q]=0.0f;
  for (int i=0;i<ITERS/4;i++){
#pragma unroll
    for (int k=0;k<4;k++)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
                   : "r"(A0), "r"(A1), "r"(A2), "r"(A3), "r"(B0), "r"(B1));
  }
  float s=0.0f; for (int k=0;k<4;k++) for (int q=0;q<4;q++) s+=c[k][q];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
int main(){
  int dev=0; cudaDeviceProp p; cudaGetDeviceProperties(&p,dev);
  printf("name=%s sms=%d l2=%d smem_optin=%zu\n", p.name, p.multiProcessorCount, p.l2CacheSize, p.sharedMemPerBlockOptin);
  int blocks=p.multiProcessorCount*8, threads=256; size_t n=(size_t)blocks*threads;
  void* buf; cudaMalloc(&buf, n*8);
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for(int rep=0;rep<2;rep++){
  cudaEventRecord(e0); k_ffma<<<blocks,threads>>>((float*)buf,0.999f,0.001f); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("ffma: %.1f TFLOP/s (fma=2)\n", 2.0*8*ITERS*n/ms/1e9);
  cudaEventRecord(e0); k_dfma<<<blocks,threads>>>((double*)buf,0.999,0.001); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("dfma: %.3f TFLOP/s (fma=2)\n", 2.0*4*(ITERS/8)*n/ms/1e9);
  cudaEventRecord(e0); k_mufu<<<blocks,threads>>>((float*)buf,0.5f); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("ex2: %.2f Tops/s\n", 4.0*(ITERS/4)*n/ms/1e9);
  cudaEventRecord(e0); k_imad<<<blocks,threads>>>((unsigned*)buf,1664525u,1013904223u); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("imad: %.1f Tops/s\n", 8.0*ITERS*n/ms/1e9);
  cudaEventRecord(e0); k_mulhi<<<blocks,threads>>>((unsigned*)buf,0xD2511F53u); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("umulhi+xor: %.1f Tpairs/s\n", 4.0*ITERS*n/ms/1e9);
  cudaEventRecord(e0); k_tanh<<<blocks,threads>>>((float*)buf,0.5f); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("tanh.f32: %.2f Tops/s\n", 4.0*(ITERS/4)*n/ms/1e9);
  cudaEventRecord(e0); k_tanh2<<<blocks,threads>>>((float*)buf,0x00010001u); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("tanh.bf16x2: %.2f Tinstr/s (2 values each)\n", 4.0*(ITERS/4)*n/ms/1e9);
  cudaEventRecord(e0); k_tanhh2<<<blocks,threads>>>((float*)buf,0x00010001u); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("tanh.f16x2: %.2f Tinstr/s (2 values each)\n", 4.0*(ITERS/4)*n/ms/1e9);
  cudaEventRecord(e0); k_ex2h2<<<blocks,threads>>>((float*)buf,0x80008000u); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("ex2.f16x2: %.2f Tinstr/s (2 values each)\n", 4.0*(ITERS/4)*n/ms/1e9);
  cudaEventRecord(e0); k_mma<<<blocks,threads>>>((float*)buf,0x3f803f80u); cudaEventRecord(e1); cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms,e0,e1); printf("mma.sync bf16 m16n8k16: %.1f TFLOP/s\n", 4096.0*4*(ITERS/4)*(n/32)/ms/1e9);
  }
  cudaError_t err=cudaGetLastError(); printf("err=%s\n", cudaGetErrorString(err));
  cudaFree(buf); return err!=cudaSuccess;
}
