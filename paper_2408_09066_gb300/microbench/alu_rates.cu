// ALU throughput microbenchmark: MUFU sin, sin+cos and ex2, FP32 FMA and FP64
// FMA per SM and clock.  These rates set the ALU roofline of the encode
// kernels (an exponential costs two MUFU operations or an FMA-pipe polynomial).
//
// Each thread runs 8 (FP64: 4) independent dependent chains of one operation
// for a fixed number of iterations over 8 CTAs of 256 threads per SM; the rate
// per SM and clock is op-instances / time / SMs / the device's clock rate.  The
// loop's own counter and branch take issue slots too, so the FMA figure reads
// below the pipe's 128 lane operations per SM and clock.
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o alu_rates alu_rates.cu && ./alu_rates
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s @%d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<int OP>
__global__ void kern(float* out, int iters, float seed) {
  float a0 = seed + threadIdx.x*1e-3f, a1=a0+0.1f,a2=a0+0.2f,a3=a0+0.3f,a4=a0+0.4f,a5=a0+0.5f,a6=a0+0.6f,a7=a0+0.7f;
  for (int i = 0; i < iters; ++i) {
    if (OP == 0) { // sin
      a0=__sinf(a0);a1=__sinf(a1);a2=__sinf(a2);a3=__sinf(a3);a4=__sinf(a4);a5=__sinf(a5);a6=__sinf(a6);a7=__sinf(a7);
    } else if (OP == 1) { // sincos pair
      float s,c; __sincosf(a0,&s,&c); a0=s+c; __sincosf(a1,&s,&c); a1=s+c; __sincosf(a2,&s,&c); a2=s+c; __sincosf(a3,&s,&c); a3=s+c;
      __sincosf(a4,&s,&c); a4=s+c; __sincosf(a5,&s,&c); a5=s+c; __sincosf(a6,&s,&c); a6=s+c; __sincosf(a7,&s,&c); a7=s+c;
    } else if (OP == 2) { // ex2
      a0=exp2f(-a0);a1=exp2f(-a1);a2=exp2f(-a2);a3=exp2f(-a3);a4=exp2f(-a4);a5=exp2f(-a5);a6=exp2f(-a6);a7=exp2f(-a7);
    } else if (OP == 3) { // fma
      a0=fmaf(a0,0.999f,0.001f);a1=fmaf(a1,0.999f,0.001f);a2=fmaf(a2,0.999f,0.001f);a3=fmaf(a3,0.999f,0.001f);
      a4=fmaf(a4,0.999f,0.001f);a5=fmaf(a5,0.999f,0.001f);a6=fmaf(a6,0.999f,0.001f);a7=fmaf(a7,0.999f,0.001f);
    }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void kern64(double* out, int iters, double seed) {
  double a0 = seed + threadIdx.x*1e-3, a1=a0+0.1,a2=a0+0.2,a3=a0+0.3;
  for (int i = 0; i < iters; ++i) { a0=fma(a0,0.999,0.001);a1=fma(a1,0.999,0.001);a2=fma(a2,0.999,0.001);a3=fma(a3,0.999,0.001); }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3;
}
int main() {
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, 0));
  int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("name=%s sms=%d cc=%d.%d clock_khz=%d smem_optin=%zu l2=%d\n", p.name, p.multiProcessorCount, p.major, p.minor, clk, p.sharedMemPerBlockOptin, p.l2CacheSize);
  int sms = p.multiProcessorCount; int blocks = sms*8, threads=256; int n = blocks*threads;
  float* out; CK(cudaMalloc(&out, n*sizeof(float)*2));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* names[4]={"sin","sincos","ex2","fma"};
  for (int op=0; op<4; ++op) {
    int iters = (op==3)? 200000 : 20000;
    for (int rep=0; rep<3; ++rep) {
      cudaEventRecord(e0);
      if(op==0) kern<0><<<blocks,threads>>>(out,iters,0.5f);
      if(op==1) kern<1><<<blocks,threads>>>(out,iters,0.5f);
      if(op==2) kern<2><<<blocks,threads>>>(out,iters,0.5f);
      if(op==3) kern<3><<<blocks,threads>>>(out,iters,0.5f);
      cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      double ops = (double)n*iters*8; // op-instances (sincos counts pairs)
      printf("%s rep%d: %.3f ms  %.3e op/s  per-SM-per-clk(@%dMHz)=%.2f\n", names[op], rep, ms, ops/(ms*1e-3), clk/1000,
             ops/(ms*1e-3)/sms/(clk*1e3));
    }
  }
  double* o64; CK(cudaMalloc(&o64, n*sizeof(double)));
  for (int rep=0; rep<2; ++rep) {
    int iters=20000;
    cudaEventRecord(e0); kern64<<<blocks,threads>>>(o64,iters,0.5); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms,e0,e1); double ops=(double)n*iters*4;
    printf("dfma rep%d: %.3f ms %.3e op/s per-SM-per-clk=%.3f\n", rep, ms, ops/(ms*1e-3), ops/(ms*1e-3)/sms/(clk*1e3));
  }
  return 0;
}
