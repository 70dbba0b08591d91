// probe_sfu.cu -- per-SM-clock issue rates of MUFU ex2/lg2, FFMA and DFMA on the
// current GPU (one CTA per SM, 8 independent chains per thread, clock64 per CTA).
// These rates give the SFU roofline of the pair kernel (see bench.py).
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_sfu probe_sfu.cu && ./probe_sfu
#include <cstdio>
#include <cuda_runtime.h>
__device__ __forceinline__ float ex2f(float x){float y; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;}
__device__ __forceinline__ float lg2f(float x){float y; asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;}
template<int MODE>
__global__ void kern(float* out, long long* cyc, int iters){
  float a[8]; for(int k=0;k<8;k++) a[k] = 0.001f*(threadIdx.x+k) - 0.5f;
  double d[8]; for(int k=0;k<8;k++) d[k] = 1e-3*(threadIdx.x+k);
  __syncthreads();
  long long t0 = clock64();
  for(int it=0; it<iters; ++it){
    #pragma unroll
    for(int k=0;k<8;k++){
      if (MODE==0) a[k] = ex2f(a[k]);                 // pure ex2 chain
      if (MODE==1) a[k] = lg2f(a[k]+2.0f);            // lg2 (+1 fadd)
      if (MODE==2) a[k] = fmaf(a[k], 0.999f, 0.001f); // ffma
      if (MODE==3) d[k] = fma(d[k], 0.999, 0.001);    // dfma
      if (MODE==4) { a[k] = ex2f(a[k]); a[k] = fmaf(a[k],0.9f,0.1f); a[k] = fmaf(a[k],0.9f,0.1f); a[k] = fmaf(a[k],0.9f,-0.5f);} // ex2 + 3 ffma
      if (MODE==5) { a[k] = ex2f(a[k]) ; a[k] = lg2f(a[k]+1.5f);} // ex2 + lg2 + fadd
    }
  }
  __syncthreads();
  long long t1 = clock64();
  float s=0; for(int k=0;k<8;k++) s+=a[k]+(float)d[k];
  if (s==123.456f) out[0]=s;
  if (threadIdx.x==0) cyc[blockIdx.x] = t1-t0;
}
int main(){
  int dev=0; cudaDeviceProp pr; cudaGetDeviceProperties(&pr, dev);
  int nsm = pr.multiProcessorCount; printf("SMs %d cc %d.%d\n", nsm, pr.major, pr.minor);
  float* out; long long* cyc; cudaMalloc(&out, 4); cudaMalloc(&cyc, 8*nsm*4);
  long long* h = new long long[nsm*4];
  const char* names[] = {"ex2","lg2+fadd","ffma","dfma","ex2+3ffma","ex2+lg2+fadd"};
  for (int mode=0; mode<6; ++mode){
    for (int threads : {256, 512, 1024}){
      int iters = (mode==3) ? 256 : 4096;
      cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
      for (int rep=0; rep<2; ++rep){
        cudaEventRecord(e0);
        switch(mode){case 0: kern<0><<<nsm,threads>>>(out,cyc,iters);break; case 1: kern<1><<<nsm,threads>>>(out,cyc,iters);break;
          case 2: kern<2><<<nsm,threads>>>(out,cyc,iters);break; case 3: kern<3><<<nsm,threads>>>(out,cyc,iters);break;
          case 4: kern<4><<<nsm,threads>>>(out,cyc,iters);break; case 5: kern<5><<<nsm,threads>>>(out,cyc,iters);break;}
        cudaEventRecord(e1); cudaEventSynchronize(e1);
      }
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      cudaMemcpy(h, cyc, 8*nsm, cudaMemcpyDeviceToHost);
      double mc=0; for(int i=0;i<nsm;i++) mc += h[i]; mc/=nsm;
      double ops = (double)threads*iters*8; // per SM (one block per SM)
      printf("%-14s thr=%4d  lane-ops/SM/clk=%7.2f  ms=%.3f  eff_clock_MHz=%.0f  err=%s\n", names[mode], threads, ops/mc, ms, mc/(ms*1e3), cudaGetErrorString(cudaGetLastError()));
    }
  }
  return 0;
}
