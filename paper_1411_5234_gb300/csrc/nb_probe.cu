// nb_probe.cu -- arithmetic-rate probe behind nb_measure_rate.
//
// The force kernels are bound by the FP32 FMA pipe (mixed path) or the FP64
// pipe (FP64 path), so their roofline needs the rate those pipes deliver on
// this part.  The probe runs independent FMA chains (packed f32x2, scalar
// FP32 or FP64) in every thread of a few CTAs per SM, records each CTA's SM
// and its start and end SM clock, and the host turns that into lanes per SM
// per clock: the FMA operations of an SM's CTAs over the cycles from the
// first start to the last end on that SM, the median over SMs.  Counting SM
// clock cycles makes the figure independent of the clock the GPU ran at.
#include "../../include/nbody_gb300.h"
#include "nb_integrator.cuh"

namespace nb {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__device__ __forceinline__ long long sm_clock() { return clock64(); }

__device__ __forceinline__ unsigned sm_id() {
  unsigned s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

// MODE 0: f32x2 FMA, 1: FP32 FMA, 2: FP64 FMA.  Each thread runs kProbeChains
// dependent chains of `iters` FMAs; the sum is stored so the chains survive.
template <int MODE>
__global__ void __launch_bounds__(kProbeThreads) k_rate(int iters, float* out,
                                                        long long* rec) {
  const long long t0 = sm_clock();
  float acc = 0.f;
  if (MODE == 0) {
    f2 x[kProbeChains];
    const f2 y = f2_pack(0.9999999f, 1.0000001f), z = f2_pack(1e-7f, -1e-7f);
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = f2_pack(threadIdx.x * 1e-3f + k, 0.5f * k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = f2_fma(x[k], y, z);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) {
      const float2 p = f2_unpack(x[k]);
      acc += p.x + p.y;
    }
  } else if (MODE == 1) {
    float x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = fmaf(x[k], 0.9999999f, 1e-7f);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc += x[k];
  } else {
    double x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], 0.9999999999, 1e-12);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    acc = static_cast<float>(s);
  }
  out[blockIdx.x * kProbeThreads + threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x] = sm_id();
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = sm_clock();
  }
}

}  // namespace

size_t probe_scratch_bytes(int ctas) {
  return sizeof(float) * (size_t)ctas * kProbeThreads + 3 * sizeof(long long) * (size_t)ctas;
}

cudaError_t launch_rate_probe(int mode, int ctas, int iters, void* scratch, cudaStream_t st) {
  float* out = static_cast<float*>(scratch);
  long long* rec = reinterpret_cast<long long*>(out + (size_t)ctas * kProbeThreads);
  if (mode == 0)
    k_rate<0><<<ctas, kProbeThreads, 0, st>>>(iters, out, rec);
  else if (mode == 1)
    k_rate<1><<<ctas, kProbeThreads, 0, st>>>(iters, out, rec);
  else
    k_rate<2><<<ctas, kProbeThreads, 0, st>>>(iters, out, rec);
  return cudaGetLastError();
}

double probe_lanes_per_launch(int mode, int ctas, int iters) {
  const double lanes_per_fma = mode == 0 ? 2.0 : 1.0;
  return lanes_per_fma * kProbeChains * (double)iters * kProbeThreads * ctas;
}

}  // namespace nb
