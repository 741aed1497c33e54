// Common device helpers for the Krylov IPM library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>

#define KQ_WARP 32

// ---------------------------------------------------------------- storage
__device__ __forceinline__ double ld_as_f64(const double *p, int64_t i) { return p[i]; }
__device__ __forceinline__ double ld_as_f64(const float *p, int64_t i) { return (double)p[i]; }
__device__ __forceinline__ double ld_as_f64(const __nv_bfloat16 *p, int64_t i) {
  return (double)__bfloat162float(p[i]);
}
__device__ __forceinline__ float ld_as_f32(const double *p, int64_t i) { return (float)p[i]; }
__device__ __forceinline__ float ld_as_f32(const float *p, int64_t i) { return p[i]; }
// store a double in the storage type (round to nearest)
__device__ __forceinline__ void st_from_f64(double *p, int64_t i, double v) { p[i] = v; }
__device__ __forceinline__ void st_from_f64(float *p, int64_t i, double v) { p[i] = (float)v; }
__device__ __forceinline__ void st_from_f64(__nv_bfloat16 *p, int64_t i, double v) {
  p[i] = __double2bfloat16(v);
}
__device__ __forceinline__ float ld_as_f32(const __nv_bfloat16 *p, int64_t i) {
  return __bfloat162float(p[i]);
}

template <class T> __device__ __forceinline__ T ld_as(const double *p, int64_t i);
template <> __device__ __forceinline__ double ld_as<double>(const double *p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ float ld_as<float>(const double *p, int64_t i) { return (float)p[i]; }

template <class T, class S> __device__ __forceinline__ T cvt(S v) { return (T)v; }

// streaming (read-once) loads: do not keep in L1
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }

// ---------------------------------------------------------------- reductions
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of NV doubles; result valid in thread 0.  `sh` needs
// 32*NV doubles.  All threads must call.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sh[k * 32 + lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double block_min(double v, double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_min(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? sh[lane] : INFINITY;
    v = warp_min(t);
  }
  __syncthreads();
  return v;
}

// ---------------------------------------------------------------- timers
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- grid barrier
// Barrier over all CTAs of a cooperative launch (or of one team of it).  The
// arrival counter only grows: the CTA that adds to it at count c waits until
// the counter reaches the next multiple of nblocks, so no CTA has to reset
// it and one release-add plus acquire-loads make the whole handshake.  Every
// wait is bounded by `budget_ns`; on expiry, or when another CTA has already
// recorded an error, the CTA records KQ_ERR_TIMEOUT-style status in *err and
// returns false (the caller then leaves its loop).  The kernel is launched
// with cudaLaunchCooperativeKernel, so all CTAs are co-resident and a
// correct program never reaches the budget.  The counter is zeroed before
// every launch.
struct GridBar {
  unsigned int *count;   // arrival counter
  unsigned int *gen;     // unused (kept for the layout of the status words)
  int *err;              // error flag (0 = ok)
  unsigned int nblocks;
  uint64_t budget_ns;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_sync(const GridBar &g) {
  __shared__ int s_ok;
  if (g.nblocks == 1) {
    // a single CTA: the CTA barrier orders its global and shared memory
    __syncthreads();
    return true;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(g.count) : "memory");
    const unsigned int target = (old / g.nblocks + 1u) * g.nblocks;
    if ((int)(ld_acquire_u32(g.count) - target) < 0) {
      const uint64_t t0 = global_ns();
      unsigned int spins = 0;
      while ((int)(ld_acquire_u32(g.count) - target) < 0) {
        if (((++spins) & 255u) == 0u) {
          if (global_ns() - t0 > g.budget_ns) { ok = 0; break; }
          if (*((volatile int *)g.err) != 0) { ok = 0; break; }
        }
      }
    }
    if (!ok) atomicCAS(g.err, 0, 7 /* KQ_ERR_TIMEOUT */);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------- misc
__device__ __forceinline__ double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

__host__ __device__ __forceinline__ int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
