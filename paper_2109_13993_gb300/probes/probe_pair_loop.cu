// probe_pair_loop.cu -- ceiling of the FP32 pair inner loop in isolation: one CTA of
// 512 threads per SM, a 96-row tile of samples resident in shared memory, no copies
// and no barriers; the same per-thread work as the pair kernel (four pairs, two
// residuals each, log cosh and u e^{-u^2/2} moments closed every 32 samples).
// Reports pair-samples per SM clock for variants of the per-sample arithmetic.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_pair_loop probe_pair_loop.cu && ./probe_pair_loop
#include <cstdio>
#include <cuda_runtime.h>
__device__ __forceinline__ float ex2a(float x){float y; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;}
__device__ __forceinline__ float lg2a(float x){float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;}
constexpr float kC3 = -3.39728720115207617088f;
constexpr int TI=64, LDS=132, CH=128, kSub=32;
struct Acc2 { float2 A, P, G; };
template<int MODE>
__device__ __forceinline__ void acc2_add(Acc2& s, float2 u) {
  if (MODE == 0) {  // current
    const float2 q = __fmul2_rn(u, u);
    float2 g; g.x = ex2a(-q.x); g.y = ex2a(-q.y);
    s.G = __ffma2_rn(u, g, s.G);
    float2 t; t.x = fabsf(u.x) * kC3; t.y = fabsf(u.y) * kC3;
    float2 e; e.x = ex2a(t.x); e.y = ex2a(t.y);
    s.P = __ffma2_rn(s.P, e, s.P);
    s.A = __fadd2_rn(s.A, t);
  } else if (MODE == 1) {  // scalar
    float qx = u.x*u.x, qy = u.y*u.y;
    float gx = ex2a(-qx), gy = ex2a(-qy);
    s.G.x = fmaf(u.x, gx, s.G.x); s.G.y = fmaf(u.y, gy, s.G.y);
    float tx = fabsf(u.x)*kC3, ty = fabsf(u.y)*kC3;
    float ex = ex2a(tx), ey = ex2a(ty);
    s.P.x = fmaf(s.P.x, ex, s.P.x); s.P.y = fmaf(s.P.y, ey, s.P.y);
    s.A.x += tx; s.A.y += ty;
  } else if (MODE == 2) {  // packed, |u| by bit ops then FMUL2
    const float2 q = __fmul2_rn(u, u);
    float2 g; g.x = ex2a(-q.x); g.y = ex2a(-q.y);
    s.G = __ffma2_rn(u, g, s.G);
    float2 au = make_float2(__uint_as_float(__float_as_uint(u.x) & 0x7fffffffu), __uint_as_float(__float_as_uint(u.y) & 0x7fffffffu));
    float2 t = __fmul2_rn(au, make_float2(kC3, kC3));
    float2 e; e.x = ex2a(t.x); e.y = ex2a(t.y);
    s.P = __ffma2_rn(s.P, e, s.P);
    s.A = __fadd2_rn(s.A, t);
  } else if (MODE == 3) {  // packed; A accumulates |u| (ALU abs), ex2 of -|y| with y formed by FMUL2 of u
    const float2 q = __fmul2_rn(u, u);
    float2 g; g.x = ex2a(-q.x); g.y = ex2a(-q.y);
    s.G = __ffma2_rn(u, g, s.G);
    float2 y = __fmul2_rn(u, make_float2(kC3, kC3));
    float2 e; e.x = ex2a(-fabsf(y.x)); e.y = ex2a(-fabsf(y.y));
    s.P = __ffma2_rn(s.P, e, s.P);
    s.A = __fadd2_rn(s.A, make_float2(fabsf(y.x), fabsf(y.y)));
  }
}
template<int MODE, int NT>
__global__ void __launch_bounds__(NT,1) kern(float* out, long long* cyc, int iters) {
  extern __shared__ float sm[];
  for (int k = threadIdx.x; k < (TI+32)*LDS; k += NT) sm[k] = 2.5f*__sinf(0.37f*k + 0.1f*blockIdx.x);
  __syncthreads();
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int TIe = NT / 8;   // rows per tile for this thread count (NT=512 -> 64)
  const float* R0 = sm + ty*LDS; const float* R1 = sm + (ty + TIe/2)*LDS;
  const float* C0 = sm + (TI + tx)*LDS; const float* C1 = sm + (TI + tx + 16)*LDS;
  float2 s2[4], sr2[4];
  for (int q = 0; q < 4; ++q) { float s = 0.9f + 0.01f*q + 1e-4f*tid; s2[q] = make_float2(s,s); sr2[q] = make_float2(-0.3f*s, -0.3f*s); }
  float D[8], Gt[8];
  for (int j=0;j<8;j++){D[j]=0.f;Gt[j]=0.f;}
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll 1
    for (int tt = 0; tt < CH; tt += kSub) {
      Acc2 acc[8];
#pragma unroll
      for (int j=0;j<8;j++){acc[j].A=make_float2(0.f,0.f);acc[j].P=make_float2(1.f,1.f);acc[j].G=make_float2(0.f,0.f);}
#pragma unroll 2
      for (int uu = 0; uu < kSub; uu += 4) {
        const float4 xr0 = *reinterpret_cast<const float4*>(R0 + tt + uu);
        const float4 xr1 = *reinterpret_cast<const float4*>(R1 + tt + uu);
        const float4 xc0 = *reinterpret_cast<const float4*>(C0 + tt + uu);
        const float4 xc1 = *reinterpret_cast<const float4*>(C1 + tt + uu);
        const float2 xi[2][2] = {{make_float2(xr0.x, xr0.y), make_float2(xr0.z, xr0.w)},{make_float2(xr1.x, xr1.y), make_float2(xr1.z, xr1.w)}};
        const float2 xj[2][2] = {{make_float2(xc0.x, xc0.y), make_float2(xc0.z, xc0.w)},{make_float2(xc1.x, xc1.y), make_float2(xc1.z, xc1.w)}};
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 vi = xi[q >> 1][h], vj = xj[q & 1][h];
            const float2 a = __ffma2_rn(s2[q], vi, __fmul2_rn(sr2[q], vj));
            const float2 bb = __ffma2_rn(s2[q], vj, __fmul2_rn(sr2[q], vi));
            acc2_add<MODE>(acc[2*q], a);
            acc2_add<MODE>(acc[2*q+1], bb);
          }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float lsum = lg2a(acc[j].P.x * acc[j].P.y);
        const float asum = acc[j].A.x + acc[j].A.y;
        D[j] += fmaf(0.693f, lsum, fmaf(asum, 0.3f, -1.0f));
        Gt[j] += acc[j].G.x + acc[j].G.y;
      }
    }
  }
  long long t1 = clock64();
  float s = 0; for (int j=0;j<8;j++) s += D[j] + Gt[j];
  out[blockIdx.x*NT + tid] = s;
  if (tid == 0) cyc[blockIdx.x] = t1 - t0;
}
template<int MODE, int NT>
void run(const char* name, int nsm, float* out, long long* cyc) {
  int iters = 200;
  size_t smem = (TI+32)*LDS*4;
  cudaFuncSetAttribute(kern<MODE,NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int rep = 0; rep < 2; ++rep) { cudaEventRecord(e0); kern<MODE,NT><<<nsm, NT, smem>>>(out, cyc, iters); cudaEventRecord(e1); cudaEventSynchronize(e1); }
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  long long h[1024]; cudaMemcpy(h, cyc, 8*nsm, cudaMemcpyDeviceToHost);
  double mc = 0; for (int i=0;i<nsm;i++) mc += h[i]; mc /= nsm;
  double ps = (double)NT*4*CH*iters;  // pair-samples per SM
  cudaFuncAttributes fa; cudaFuncGetAttributes(&fa, kern<MODE,NT>);
  printf("%-28s NT=%4d regs=%3d spill=%zu  pair-samples/clk/SM=%6.3f  (%.1f%% of 7.76)  ms=%.3f  err=%s\n", name, NT, fa.numRegs, fa.localSizeBytes, ps/mc, 100*ps/mc/7.76, ms, cudaGetErrorString(cudaGetLastError()));
}
int main() {
  cudaDeviceProp pr; cudaGetDeviceProperties(&pr, 0);
  int nsm = pr.multiProcessorCount;
  float* out; long long* cyc; cudaMalloc(&out, 4*nsm*1024); cudaMalloc(&cyc, 8*nsm);
  run<0,512>("packed, t = |u| kC3", nsm, out, cyc);
  run<1,512>("scalar", nsm, out, cyc);
  run<2,512>("packed, abs by bit-and", nsm, out, cyc);
  run<3,512>("packed, ex2(-|y|) (the kernel)", nsm, out, cyc);
  run<0,256>("packed, t = |u| kC3", nsm, out, cyc);
  run<1,256>("scalar", nsm, out, cyc);
  return 0;
}
