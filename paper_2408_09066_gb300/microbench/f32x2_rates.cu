// Packed FP32 throughput: fma.rn.f32x2 (two FMAs per instruction) alone, and
// beside MUFU sines in the same loop (4 sines with 8 or 16 packed FMAs per
// iteration), per SM and clock.  The encode does its FMA-pipe work in packed
// f32x2 form and runs it beside MUFU sin/cos.
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o f32x2_rates f32x2_rates.cu && ./f32x2_rates
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s @%d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)
__device__ __forceinline__ unsigned long long pk(float a, float b){unsigned long long r; asm("mov.b64 %0, {%1,%2};":"=l"(r):"f"(a),"f"(b)); return r;}
__device__ __forceinline__ float lo(unsigned long long r){float a,b; asm("mov.b64 {%0,%1}, %2;":"=f"(a),"=f"(b):"l"(r)); return a+b;}
#define F2(x, m, c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x) : "l"(m), "l"(c))
template<int MODE> __global__ void kern(float* out, int iters, float seed) {
  float s = seed + threadIdx.x * 1e-3f;
  unsigned long long m = pk(0.999f, 0.998f), c = pk(0.001f, 0.002f);
  unsigned long long x0=pk(s,s+1),x1=pk(s+2,s+3),x2=pk(s+4,s+5),x3=pk(s+6,s+7),x4=pk(s+8,s+9),x5=pk(s+10,s+11),x6=pk(s+12,s+13),x7=pk(s+14,s+15);
  float a0=s,a1=s+.1f,a2=s+.2f,a3=s+.3f;
  for (int i = 0; i < iters; ++i) {
    if (MODE == 0) { F2(x0,m,c);F2(x1,m,c);F2(x2,m,c);F2(x3,m,c);F2(x4,m,c);F2(x5,m,c);F2(x6,m,c);F2(x7,m,c); }
    if (MODE == 1) { // 4 MUFU sin + 8 packed FMA
      a0=__sinf(a0);a1=__sinf(a1);a2=__sinf(a2);a3=__sinf(a3);
      F2(x0,m,c);F2(x1,m,c);F2(x2,m,c);F2(x3,m,c);F2(x4,m,c);F2(x5,m,c);F2(x6,m,c);F2(x7,m,c); }
    if (MODE == 2) { // 4 MUFU sin + 16 packed FMA
      a0=__sinf(a0);a1=__sinf(a1);a2=__sinf(a2);a3=__sinf(a3);
      F2(x0,m,c);F2(x1,m,c);F2(x2,m,c);F2(x3,m,c);F2(x4,m,c);F2(x5,m,c);F2(x6,m,c);F2(x7,m,c);
      F2(x0,m,c);F2(x1,m,c);F2(x2,m,c);F2(x3,m,c);F2(x4,m,c);F2(x5,m,c);F2(x6,m,c);F2(x7,m,c); }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = lo(x0)+lo(x1)+lo(x2)+lo(x3)+lo(x4)+lo(x5)+lo(x6)+lo(x7)+a0+a1+a2+a3;
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0)); int sms=p.multiProcessorCount;
  int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  int blocks=sms*8, threads=256, n=blocks*threads; float* out; CK(cudaMalloc(&out,n*4));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* nm[3]={"ffma2 x8","sin x4 + ffma2 x8","sin x4 + ffma2 x16"};
  for(int mode=0;mode<3;++mode) for(int rep=0;rep<2;++rep){
    int iters = 20000;
    cudaEventRecord(e0);
    if(mode==0)kern<0><<<blocks,threads>>>(out,iters,.5f);
    if(mode==1)kern<1><<<blocks,threads>>>(out,iters,.5f);
    if(mode==2)kern<2><<<blocks,threads>>>(out,iters,.5f);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); CK(cudaGetLastError());
    float ms; cudaEventElapsedTime(&ms,e0,e1);
    double it=(double)n*iters; double clkhz=clk*1e3;
    printf("%-20s rep%d %.3f ms: per SM-clk: packed-FMA instr-lanes=%.1f (flop-lanes %.1f)\n", nm[mode], rep, ms,
      it*(mode==2?16:8)/(ms*1e-3)/sms/clkhz, 2*it*(mode==2?16:8)/(ms*1e-3)/sms/clkhz);
  }
  return 0;
}
