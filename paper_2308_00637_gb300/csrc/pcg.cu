// Persistent Jacobi-PCG on the doubly augmented KKT system (Eq. (9)).
//
//   K = [ Q + 2 B'D^-1 B   B' ]      Q = H + diag(dg),  B = [C; A_L; -A_U]
//       [ B                D  ]      D = diag(mu 1, S_lA/Lam_lA, S_uA/Lam_uA)
//
// K is never formed (section 3.2): one product K p is a single pass over the
// rows of the operator.  For a general row i with t_i = A_i p_x,
//     top    += A_i' (2 t_i (1/D_li + 1/D_ui) + p_li - p_ui)
//     bottom  = ( t_i + D_li p_li,  -t_i + D_ui p_ui )
// so A is read once per product (two-sided rows folded).  For the dose
// structure (H = 2 P'WP, A = scaled rows of P) the H and A parts share the
// same read of P.
//
// One cooperative launch runs the whole PCG solve.  Per iteration:
//   phase A  : q = K p, with p = y + beta p_old formed on the fly (so the
//              search direction update needs no barrier of its own), and the
//              partial sums of p'q (p'Aq terms by linearity: p_x'A' c = c't);
//   barrier  : alpha = rho / p'q;
//   phase C  : z += alpha p, r -= alpha q, y = r / diag(K), partial |r|^2, r'y;
//   barrier  : beta = rho'/rho, convergence test |r| <= tol |rhs|.
// Dots are FP64 and summed in a fixed order (deterministic).  Every barrier
// wait is bounded; on expiry the kernel records a status and returns.
#include "common.cuh"
#include "kq_internal.h"
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>
#include <type_traits>

namespace {

struct PcgArgs {
  DevProb P;
  const double *Dl, *Du, *cl, *cu, *dg, *diag;
  double mu;
  const double *rhs;   // right-hand side (SOLVE) or the vector v (APPLY)
  double *z;           // solution (SOLVE) or K v (APPLY)
  double *r, *y, *pb0, *pb1, *qlam;
  void *accx;
  double *g;
  double *slots;
  const int64_t *row_begin;
  const int32_t *win_lo, *win_hi;
  int win_cap;
  GridBar bar;
  double tol2;
  int maxit;
  int apply;
  int *iters;
  double *resn;
  // CSR staging (bulk async copies of row chunks into shared memory)
  const ChunkInfo *chunks;      // all chunks, CTA-major
  const int32_t *cta_chunk;     // G+1 chunk ranges
  const RowDesc *rdesc;         // row descriptors, chunk-major
  const int32_t *a_lo, *a_hi;   // G ranges of A rows owned by each CTA's P rows
  int a_cap, ch_cap, desc_cap, tab_cap;
  int copy_piece;               // bytes per bulk copy (multiple of 16)
  int stages;                   // shared-memory ring depth
  int producer;                 // 0: per-thread cp.async, 1: bulk copies + mbarrier
  int stag_window;              // >0: stop when |r| has not halved over this many iterations
  double *coefA;                // dense: per-row coefficients of the column pass (m)
  // register-streamed CSR (FP32 products)
  const RowSlot *rslot;
  const float4 *rval4;
  const uint2 *rcol2;           // four 16-bit window-relative columns per lane
  const float *rw2lo;           // per P row: 2 sigma w - (float)(2 sigma w) (FP64 products)
  int rws;                      // per-warp accumulator stride (floats, multiple of 32)
  int pf_dist;                  // L2 prefetch distance in warp steps (0: off, the default)
  double *dinv;                 // 1 / diag(K), formed at the start of a solve (or null)
  float *p32_0, *p32_1, *y32;   // FP32 copies of p (paired with pb0 / pb1) and y (or null)
  double *lanczos;              // (alpha_j, beta_j) per iteration, or null (not recorded)
  int lanczos_cap;              // iterations that fit in lanczos
  int run;                      // batched launches: 0 = skip this problem
  int colpass_min_n;            // dense: column-blocked A' pass from this n on (0: 512)
};

// barrier parameter of the problem (device-side in the batched solver's graph)
__device__ __forceinline__ double mu_of(const PcgArgs &a) { return a.P.mu_dev ? *a.P.mu_dev : a.mu; }

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }


// Threads that update the owned vector entries: one entry per thread where
// the block allows, on as few warps as that takes.  The SM's FP64 pipe is
// narrow, so warps without entries stay out of the FP64 reductions.
__device__ __forceinline__ int vec_threads(int64_t owned) {
  int64_t w = (owned + 31) & ~(int64_t)31;
  if (w < 32) w = 32;
  if (w > (int64_t)blockDim.x) w = blockDim.x;
  return (int)w;
}

// FP32 copy of p paired with a given FP64 buffer (null when not kept)
__device__ __forceinline__ float *p32_of(const PcgArgs &a, const double *pbuf) {
  if (!a.p32_0) return nullptr;
  return pbuf == a.pb0 ? a.p32_0 : a.p32_1;
}

// p_new for this CTA's owned vector entries; returns sum dg_j p_j^2 (x part)
__device__ __forceinline__ double write_owned_p(const PcgArgs &a, const double *ysrc,
                                                const double *pold, double *pnew, double beta,
                                                int64_t vb, int64_t ve) {
  double pq = 0.0;
  const int64_t n = a.P.n;
  const int vt = vec_threads(ve - vb);
  float *p32 = a.apply ? nullptr : p32_of(a, pnew);
  if ((int)threadIdx.x < vt) {
    for (int64_t i = vb + threadIdx.x; i < ve; i += vt) {
      double pi = ldcg(ysrc + i) + beta * ldcg(pold + i);
      pnew[i] = pi;
      if (p32) p32[i] = (float)pi;
      if (i < n) pq += a.dg[i] * pi * pi;
    }
  }
  return pq;
}

// Sum over the vector threads (warps 0 .. vt/32-1) of NV doubles; result in
// thread 0.  All threads must call.
template <int NV>
__device__ __forceinline__ void vec_sum(double (&v)[NV], double *sh, int vt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwv = (vt + 31) >> 5;
  if (wid < nwv) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (int w = 0; w < nwv; ++w) t += sh[k * 32 + w];
      v[k] = t;
    }
  }
  __syncthreads();
}

// Block sum of one double held by any thread, through a shared buffer of
// blockDim doubles: four warps add a quarter each, thread 0 the four partials.
__device__ __forceinline__ double block_sum_buf(double v, double *buf, double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nt = blockDim.x;
  buf[threadIdx.x] = v;
  __syncthreads();
  const int np = min(4, (nt + 31) >> 5), nq = (nt + np - 1) / np;
  if (wid < np) {
    double t = 0.0;
    for (int j = wid * nq + lane; j < min(nt, (wid + 1) * nq); j += 32) t += buf[j];
    t = warp_sum(t);
    if (lane == 0) sh[wid] = t;
  }
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < np; ++w) r += sh[w];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- DENSE (explicit H, dense A, C)
// Eight consecutive entries of a row as T (16-byte loads; the caller checks
// that the address is aligned to 8 entries).
template <class S, class T> struct Load8;
template <class T> struct Load8<__nv_bfloat16, T> {
  static __device__ __forceinline__ void run(const __nv_bfloat16 *p, T (&v)[8]) {
    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
    const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(b[k]);
      v[2 * k] = (T)f.x;
      v[2 * k + 1] = (T)f.y;
    }
  }
};
template <class T> struct Load8<float, T> {
  static __device__ __forceinline__ void run(const float *p, T (&v)[8]) {
    const float4 x = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 y = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = (T)x.x; v[1] = (T)x.y; v[2] = (T)x.z; v[3] = (T)x.w;
    v[4] = (T)y.x; v[5] = (T)y.y; v[6] = (T)y.z; v[7] = (T)y.w;
  }
};
template <class T> struct Load8<double, T> {
  static __device__ __forceinline__ void run(const double *p, T (&v)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 x = __ldg(reinterpret_cast<const double2 *>(p) + k);
      v[2 * k] = (T)x.x;
      v[2 * k + 1] = (T)x.y;
    }
  }
};

// dot of one row with the p window; vectorised when the rows are 8-aligned
template <class S, class T>
__device__ __forceinline__ T row_dot(const S *r, const T *pw, int64_t n, bool vec, int lane) {
  T dot = (T)0;
  if (vec) {
    for (int64_t j = 8 * lane; j < n; j += 256) {
      T v[8];
      Load8<S, T>::run(r + j, v);
#pragma unroll
      for (int k = 0; k < 8; ++k) dot += v[k] * pw[j + k];   // pw is zero beyond n
    }
  } else {
    for (int64_t j = lane; j < n; j += 32) dot += (T)ld_as_f64(r, j) * pw[j];
  }
  return warp_sum(dot);
}

// dots of two rows with the p window (the second row optional): both rows'
// loads are in flight together
template <class S, class T>
__device__ __forceinline__ void row_dot2(const S *r0, const S *r1, bool two, const T *pw, int64_t n,
                                         bool vec, int lane, T &d0, T &d1) {
  d0 = (T)0;
  d1 = (T)0;
  if (vec) {
#pragma unroll 2
    for (int64_t j = 8 * lane; j < n; j += 256) {
      T v0[8], v1[8];
      Load8<S, T>::run(r0 + j, v0);
      if (two) Load8<S, T>::run(r1 + j, v1);
#pragma unroll
      for (int k = 0; k < 8; ++k) d0 += v0[k] * pw[j + k];
      if (two) {
#pragma unroll
        for (int k = 0; k < 8; ++k) d1 += v1[k] * pw[j + k];
      }
    }
  } else {
    for (int64_t j = lane; j < n; j += 32) {
      d0 += (T)ld_as_f64(r0, j) * pw[j];
      if (two) d1 += (T)ld_as_f64(r1, j) * pw[j];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d0 += __shfl_xor_sync(0xffffffffu, d0, o);
    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
  }
}

// ---- double-float products (FP64-class accuracy on the FP32 pipe)
// GB300 retires FP32 multiply-adds at ~64x its FP64 rate.  Where the matrix
// is stored in bf16 or f32 (exact in FP32), an FP64 product p = M v is formed
// as follows: v splits into v_h + v_l (two floats), each term m v_h is an
// exact float pair (the rounded product and its FMA residual), and every
// lane accumulates in a float pair (s_h, s_l) whose high part takes the
// rounded products through an error-free two-sum (Knuth) and whose low part
// collects the residuals, the m v_l terms and the two-sum errors.  Relative
// accuracy about 2^-48 per term (FP64: 2^-53), far inside the 1e-7 PCG
// tolerance.  The explicit _rn intrinsics keep the compiler from contracting
// a product into the following sum, which would break the error-free steps.
struct DFAcc {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add_prod(float m, float vh, float vl) {
    const float p = __fmul_rn(m, vh);
    const float e = __fmaf_rn(m, vh, -p);
    const float q = __fmaf_rn(m, vl, e);
    const float s = __fadd_rn(h, p);
    const float bp = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    l = __fadd_rn(l, __fadd_rn(err, q));
    h = s;
  }
  __device__ __forceinline__ void add(float oh, float ol) {
    const float s = __fadd_rn(h, oh);
    const float bp = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(oh, bp));
    l = __fadd_rn(l, __fadd_rn(err, ol));
    h = s;
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
      add(oh, ol);
    }
  }
  __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};

__device__ __forceinline__ void df_split(double v, float &vh, float &vl) {
  vh = __double2float_rn(v);
  vl = __double2float_rn(v - (double)vh);
}

// dots of two rows (bf16 or f32 storage) with the window held as float pairs
template <class S>
__device__ __forceinline__ void row_dot2_df(const S *r0, const S *r1, bool two, const float *ph,
                                            const float *pl, int64_t n, bool vec, int lane,
                                            double &d0, double &d1) {
  DFAcc a0, a1;
  if (vec) {
#pragma unroll 2
    for (int64_t j = 8 * lane; j < n; j += 256) {
      float v0[8], v1[8];
      Load8<S, float>::run(r0 + j, v0);
      if (two) Load8<S, float>::run(r1 + j, v1);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float xh = ph[j + k], xl = pl[j + k];
        a0.add_prod(v0[k], xh, xl);
        if (two) a1.add_prod(v1[k], xh, xl);
      }
    }
  } else {
    for (int64_t j = lane; j < n; j += 32) {
      const float xh = ph[j], xl = pl[j];
      a0.add_prod(ld_as_f32(r0, j), xh, xl);
      if (two) a1.add_prod(ld_as_f32(r1, j), xh, xl);
    }
  }
  a0.warp_reduce();
  a1.warp_reduce();
  d0 = a0.value();
  d1 = two ? a1.value() : 0.0;
}

template <class HS, class AS, class T>
struct DenseDF {
  static constexpr bool value = sizeof(T) == 8 && !std::is_same<HS, double>::value &&
                                std::is_same<AS, float>::value;
};

template <class HS, class AS>
struct OpDense {
  // vcta / vG: this CTA's rank and the number of CTAs working on the problem
  // (the whole grid for a single problem, a team in the batched solver).
  // For n >= 512 the A' part is a second, column-blocked pass over A after a
  // barrier (register accumulation, no shared-memory atomics); small problems
  // scatter each row's coefficient with shared atomics in the same pass.
  template <class T>
  static __device__ double phaseA(const PcgArgs &a, const double *ysrc, const double *pold,
                                  double *pnew, double beta, int64_t vb, int64_t ve,
                                  unsigned char *smem, int vcta, int vG, bool &ok) {
    const DevProb &P = a.P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    const int64_t n = P.n, m = P.m, me = P.me;
    const int64_t hld = P.hld > 0 ? P.hld : n, ald = P.ald > 0 ? P.ald : n;
    const int64_t npad = (n + 7) & ~(int64_t)7;
    T *pw = reinterpret_cast<T *>(smem);
    T *acc = pw + a.win_cap;
    T *accg = reinterpret_cast<T *>(a.accx);
    const HS *Hd = reinterpret_cast<const HS *>(P.Hd);
    const AS *Ad = reinterpret_cast<const AS *>(P.Ad);
    const bool hvec = (hld % 8 == 0) && ((reinterpret_cast<uintptr_t>(Hd) & 15) == 0);
    const bool avec = (ald % 8 == 0) && ((reinterpret_cast<uintptr_t>(Ad) & 15) == 0);
    // general rows handled here only when A is dense (a CSR A has its own pass)
    const int64_t md = P.akind == KQ_A_DENSE ? m : 0;
    constexpr bool DF = DenseDF<HS, AS, T>::value;
    // double-float products always take the column pass: the row-wise A'
    // scatter would need FP64 shared-memory atomics per element
    const bool colpass = (DF || n >= (a.colpass_min_n > 0 ? a.colpass_min_n : 512)) && md > 0 &&
                         a.coefA != nullptr && avec;
    // DF: the window as float pairs in the same bytes (high parts, then low)
    float *pwh = reinterpret_cast<float *>(pw), *pwl = pwh + a.win_cap;
    auto pw_at = [&](int64_t j) -> T {
      if constexpr (DF) return (T)((double)pwh[j] + (double)pwl[j]);
      else return pw[j];
    };
    double pq = write_owned_p(a, ysrc, pold, pnew, beta, vb, ve);
    for (int64_t j = tid; j < npad; j += blockDim.x) {
      const double v = j < n ? ldcg(ysrc + j) + beta * ldcg(pold + j) : 0.0;
      if constexpr (DF) df_split(v, pwh[j], pwl[j]);
      else pw[j] = (T)v;
      acc[j] = (T)0;
    }
    __syncthreads();
    const int64_t gw0 = (int64_t)vcta * nw + warp, GW = (int64_t)vG * nw;
    const int64_t lo_off = n + me, up_off = n + me + m;
    // H rows, two per warp step
    for (int64_t row = gw0; row < n; row += 2 * GW) {
      const int64_t r2 = row + GW;
      const bool two = r2 < n;
      T d0, d1;
      if constexpr (DF) {
        double e0, e1;
        row_dot2_df<HS>(Hd + row * hld, Hd + (two ? r2 : row) * hld, two, pwh, pwl, n, hvec, lane,
                        e0, e1);
        d0 = e0;
        d1 = e1;
      } else {
        row_dot2<HS, T>(Hd + row * hld, Hd + (two ? r2 : row) * hld, two, pw, n, hvec, lane, d0, d1);
      }
      if (lane == 0) {
        d0 *= (T)P.hscale;
        atomicAdd(acc + row, d0);
        pq += (ldcg(ysrc + row) + beta * ldcg(pold + row)) * (double)d0;
        if (two) {
          d1 *= (T)P.hscale;
          atomicAdd(acc + r2, d1);
          pq += (ldcg(ysrc + r2) + beta * ldcg(pold + r2)) * (double)d1;
        }
      }
    }
    // A rows, two per warp step: t = rho A_i p, coefficient, bottom entries
    auto arow = [&](int64_t ai, T dot) {
      const bool hl = P.hasl[ai] != 0, hu = P.hasu[ai] != 0;
      if (!hl && !hu) {
        if (lane == 0) {
          a.qlam[me + ai] = 0.0;
          a.qlam[me + m + ai] = 0.0;
          if (colpass) a.coefA[ai] = 0.0;
        }
        return;
      }
      const double rho_a = P.rhoA[ai];
      const double t = rho_a * (double)dot;
      const double pl = hl ? ldcg(ysrc + lo_off + ai) + beta * ldcg(pold + lo_off + ai) : 0.0;
      const double pu = hu ? ldcg(ysrc + up_off + ai) + beta * ldcg(pold + up_off + ai) : 0.0;
      const double coef = 2.0 * t * (a.cl[ai] + a.cu[ai]) + pl - pu;
      if (colpass) {
        if (lane == 0) a.coefA[ai] = coef * rho_a;
      } else {
        const T cf = (T)(coef * rho_a);
        const AS *ar = Ad + ai * ald;
        for (int64_t j = lane; j < n; j += 32) atomicAdd(acc + j, cf * (T)ld_as_f64(ar, j));
      }
      if (lane == 0) {
        const double ql = hl ? t + a.Dl[ai] * pl : 0.0;
        const double qu = hu ? -t + a.Du[ai] * pu : 0.0;
        a.qlam[me + ai] = ql;
        a.qlam[me + m + ai] = qu;
        pq += coef * t + pl * ql + pu * qu;
      }
    };
    // warps continue the global row numbering after the H rows
    const int64_t a0 = ((gw0 - n) % GW + GW) % GW;   // first A row of this warp
    for (int64_t ai = a0; ai < md; ai += 2 * GW) {
      const int64_t a2 = ai + GW;
      const bool two = a2 < md;
      T d0, d1;
      if constexpr (DF) {
        double e0, e1;
        row_dot2_df<AS>(Ad + ai * ald, Ad + (two ? a2 : ai) * ald, two, pwh, pwl, n, avec, lane,
                        e0, e1);
        d0 = e0;
        d1 = e1;
      } else {
        row_dot2<AS, T>(Ad + ai * ald, Ad + (two ? a2 : ai) * ald, two, pw, n, avec, lane, d0, d1);
      }
      arow(ai, d0);
      if (two) arow(a2, d1);
    }
    // equality rows
    const int64_t e0 = ((gw0 - n - m) % GW + GW) % GW;
    for (int64_t e = e0; e < me; e += GW) {
      const double *cr = P.Cd + e * n;
      T dot = (T)0;
      for (int64_t j = lane; j < n; j += 32) dot += (T)cr[j] * pw_at(j);
      dot = warp_sum(dot);
      const double t = (double)dot;
      const double pe = ldcg(ysrc + n + e) + beta * ldcg(pold + n + e);
      const double coef = 2.0 * t / mu_of(a) + pe;
      const T cf = (T)coef;
      for (int64_t j = lane; j < n; j += 32) atomicAdd(acc + j, cf * (T)cr[j]);
      if (lane == 0) {
        const double qe = t + mu_of(a) * pe;
        a.qlam[e] = qe;
        pq += coef * t + pe * qe;
      }
    }
    __syncthreads();
    for (int64_t j = tid; j < n; j += blockDim.x) {
      const T v = acc[j];
      if (v != (T)0) atomicAdd(accg + j, v);
    }
    if (colpass) {
      // A' (rho coef): tasks = (256-column block) x (slice of rows)
      ok = grid_sync(a.bar);
      if (!ok) return 0.0;
      const int64_t nblk = (n + 255) / 256;
      int64_t nrs = (4 * GW + nblk - 1) / nblk;
      nrs = nrs < 1 ? 1 : (nrs > md ? md : nrs);
      const int64_t rows_per = (md + nrs - 1) / nrs;
      for (int64_t task = gw0; task < nblk * nrs; task += GW) {
        const int64_t blk = task % nblk, rs = task / nblk;
        const int64_t c0 = blk * 256 + 8 * lane;
        const int64_t a0 = rs * rows_per, a1 = (a0 + rows_per < md) ? a0 + rows_per : md;
        if constexpr (DF) {
          // A' columns in double-float: the coefficient splits, A is f32
          if (c0 < n) {
            DFAcc s8[8];
            for (int64_t ai = a0; ai < a1; ++ai) {
              const double cfd = __ldcg(a.coefA + ai);
              if (cfd == 0.0) continue;
              float ch, cl;
              df_split(cfd, ch, cl);
              float v[8];
              Load8<AS, float>::run(Ad + ai * ald + c0, v);
#pragma unroll
              for (int k = 0; k < 8; ++k) s8[k].add_prod(v[k], ch, cl);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const double v = s8[k].value();
              if (c0 + k < n && v != 0.0) atomicAdd(accg + c0 + k, (T)v);
            }
          }
          continue;
        }
        T s8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) s8[k] = (T)0;
        if (c0 < n) {
          for (int64_t ai = a0; ai < a1; ++ai) {
            const T cf = (T)__ldcg(a.coefA + ai);
            if (cf == (T)0) continue;
            T v[8];
            Load8<AS, T>::run(Ad + ai * ald + c0, v);
#pragma unroll
            for (int k = 0; k < 8; ++k) s8[k] += cf * v[k];
          }
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (c0 + k < n && s8[k] != (T)0) atomicAdd(accg + c0 + k, s8[k]);
        }
      }
    }
    return pq;
  }
};

// ---------------------------------------------------------------- LOWRANK (H = Z Z', equality rows C)
template <class ZS>
struct OpLowrank {
  template <class T>
  static __device__ double phaseA(const PcgArgs &a, const double *ysrc, const double *pold,
                                  double *pnew, double beta, int64_t vb, int64_t ve,
                                  unsigned char *smem, bool &ok) {
    const DevProb &P = a.P;
    const int cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    const int64_t n = P.n, k = P.k, me = P.me, kk = k + me;
    const ZS *Z = reinterpret_cast<const ZS *>(P.Z);
    T *accg = reinterpret_cast<T *>(a.accx);
    double *ps = reinterpret_cast<double *>(smem);          // p for this CTA's rows
    double pq = write_owned_p(a, ysrc, pold, pnew, beta, vb, ve);
    const int64_t r0 = a.row_begin[cta], r1 = a.row_begin[cta + 1];
    for (int64_t i = r0 + tid; i < r1; i += blockDim.x)
      ps[i - r0] = ldcg(ysrc + i) + beta * ldcg(pold + i);
    __syncthreads();
    // phase A1: g = [Z C']' p_x  (partial over this CTA's rows)
    for (int64_t c = tid; c < kk; c += blockDim.x) {
      T s = (T)0;
      if (c < k) {
        for (int64_t i = r0; i < r1; ++i) s += (T)ld_as_f64(Z, i * k + c) * (T)ps[i - r0];
      } else {
        const double *cr = P.Cd + (c - k) * n;
        for (int64_t i = r0; i < r1; ++i) s += (T)cr[i] * (T)ps[i - r0];
      }
      atomicAdd(a.g + c, (double)s);
    }
    ok = grid_sync(a.bar);
    if (!ok) return 0.0;
    // phase A2: (Z g)_i + sum_e C_ei (2 t_e / mu + p_e)
    double *cf = ps + a.win_cap;                          // me coefficients
    T *gs = reinterpret_cast<T *>(cf + me + 1);           // g = [Z C']'p_x
    // g = [Z C']'p_x, the Z part weighted by sigma zw
    for (int64_t c = tid; c < kk; c += blockDim.x)
      gs[c] = (T)(__ldcg(a.g + c) * (c < k ? P.hscale * (P.zw ? P.zw[c] : 1.0) : 1.0));
    for (int64_t e = tid; e < me; e += blockDim.x) {
      const double t = __ldcg(a.g + k + e);
      const double pe = ldcg(ysrc + n + e) + beta * ldcg(pold + n + e);
      cf[e] = 2.0 * t / mu_of(a) + pe;
      if (cta == 0) {
        const double qe = t + mu_of(a) * pe;
        a.qlam[e] = qe;
        pq += pe * qe;
      }
    }
    __syncthreads();
    for (int64_t i = r0 + warp; i < r1; i += nw) {
      T s = (T)0;
      for (int64_t c = lane; c < k; c += 32) s += (T)ld_as_f64(Z, i * k + c) * gs[c];
      s = warp_sum(s);
      if (lane == 0) {
        double hz = (double)s;
        if (P.d0) hz += P.hscale * P.d0[i] * ps[i - r0];   // diagonal H0
        for (int64_t e = 0; e < me; ++e) hz += P.Cd[e * n + i] * cf[e];
        if (P.akind == KQ_A_CSR) atomicAdd(accg + i, (T)hz);   // shared with the A-row scatter
        else accg[i] = (T)hz;
        pq += ps[i - r0] * hz;
      }
    }
    return pq;
  }
};

// ---------------------------------------------------------------- CSR, staged through shared memory
// The CTA's rows of P are cut into chunks (host, once per problem).  Thread 0
// streams the chunks' values, columns and row descriptors into a ring of
// `stages` shared-memory stages with 1-D bulk asynchronous copies completing
// on an mbarrier per stage; the ring keeps running across PCG iterations (the
// matrix does not change, only p), so the first chunks of the next product
// are already in flight during the grid barriers.  Warps take one row each
// from the staged chunk: dot with the p window, coefficient, scatter into
// the shared accumulator.  Every mbarrier wait is bounded.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// per-thread 16-byte asynchronous copies (LSU path), grouped per chunk
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
  }
}

struct PipeState {
  uint32_t seq_issue = 0, seq_cons = 0;
  int nc = 0, c0 = 0;
};

struct OpCsrStaged {
  static __device__ __forceinline__ CsrLayout lay(const PcgArgs &a) {
    return csr_layout(a.win_cap, a.a_cap, a.ch_cap, a.desc_cap, a.tab_cap, a.stages);
  }

  // thread 0: start the copy of chunk number seq_issue (mod nc) into its stage
  static __device__ void issue_chunk(const PcgArgs &a, unsigned char *smem, const CsrLayout &L,
                                     const PipeState &ps) {
    const int j = (int)(ps.seq_issue % (uint32_t)ps.nc);
    const ChunkInfo ci = (j < a.tab_cap) ? reinterpret_cast<const ChunkInfo *>(smem + L.tab)[j]
                                         : a.chunks[ps.c0 + j];
    const int st = (int)(ps.seq_issue % (uint32_t)a.stages);
    unsigned char *sb = smem + L.stage0 + (size_t)st * L.stage_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar) + st;
    const uint32_t bytes = (uint32_t)ci.ndesc * 16u + (ci.nelem > 0 ? (uint32_t)ci.nelem * 8u : 0u);
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(sb + L.desc_off, a.rdesc + ci.desc0, (uint32_t)ci.ndesc * 16u, bar);
    if (ci.nelem > 0) {
      // split into pieces of copy_piece bytes (a multiple of 16): several
      // smaller copies keep more requests in flight than one large one
      const uint32_t total = (uint32_t)ci.nelem * 4u, piece = (uint32_t)a.copy_piece;
      for (uint32_t o = 0; o < total; o += piece) {
        const uint32_t nb = min(piece, total - o);
        bulk_g2s(sb + L.val_off + o, reinterpret_cast<const unsigned char *>(a.P.val + ci.src) + o, nb, bar);
        bulk_g2s(sb + L.col_off + o, reinterpret_cast<const unsigned char *>(a.P.col + ci.src) + o, nb, bar);
      }
    }
  }

  // all threads: copy chunk number seq_issue (mod nc) into its stage with
  // 16-byte cp.async pieces, one commit group per chunk
  static __device__ void issue_chunk_lsu(const PcgArgs &a, unsigned char *smem, const CsrLayout &L,
                                         const PipeState &ps) {
    const int j = (int)(ps.seq_issue % (uint32_t)ps.nc);
    const ChunkInfo ci = (j < a.tab_cap) ? reinterpret_cast<const ChunkInfo *>(smem + L.tab)[j]
                                         : a.chunks[ps.c0 + j];
    const int st = (int)(ps.seq_issue % (uint32_t)a.stages);
    unsigned char *sb = smem + L.stage0 + (size_t)st * L.stage_bytes;
    const int nv = ci.nelem > 0 ? ci.nelem >> 2 : 0;   // 16-byte pieces of val (and of col)
    const int nd = ci.ndesc;                            // 16-byte descriptors
    const float4 *gv = reinterpret_cast<const float4 *>(a.P.val + ci.src);
    const int4 *gc = reinterpret_cast<const int4 *>(a.P.col + ci.src);
    const int4 *gd = reinterpret_cast<const int4 *>(a.rdesc + ci.desc0);
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
      cp_async16(sb + L.val_off + 16 * (size_t)q, gv + q);
      cp_async16(sb + L.col_off + 16 * (size_t)q, gc + q);
    }
    for (int q = threadIdx.x; q < nd; q += blockDim.x) cp_async16(sb + L.desc_off + 16 * (size_t)q, gd + q);
    cp_async_commit();
  }

  // bounded wait for the copy of sequence number seq; false on timeout
  static __device__ bool wait(const PcgArgs &a, unsigned char *smem, const CsrLayout &L,
                              uint32_t seq) {
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar) + (seq % (uint32_t)a.stages);
    const uint32_t par = (seq / (uint32_t)a.stages) & 1u;
    if (mbar_try_wait(bar, par)) return true;
    const uint64_t t0 = global_ns();
    unsigned spins = 0;
    while (!mbar_try_wait(bar, par)) {
      if (((++spins) & 63u) == 0u && global_ns() - t0 > a.bar.budget_ns) return false;
    }
    return true;
  }

  template <class T>
  static __device__ void begin(const PcgArgs &a, unsigned char *smem, PipeState &ps) {
    const CsrLayout L = lay(a);
    const int cta = blockIdx.x, tid = threadIdx.x;
    ps.c0 = a.cta_chunk[cta];
    ps.nc = a.cta_chunk[cta + 1] - ps.c0;
    ps.seq_issue = ps.seq_cons = 0;
    if (tid == 0) {
      for (int s = 0; s < a.stages; ++s) mbar_init(reinterpret_cast<uint64_t *>(smem + L.bar) + s, 1);
      fence_mbar_init();
    }
    ChunkInfo *tab = reinterpret_cast<ChunkInfo *>(smem + L.tab);
    for (int j = tid; j < min(ps.nc, a.tab_cap); j += blockDim.x) tab[j] = a.chunks[ps.c0 + j];
    const int alo = a.a_lo[cta], na = min(a.a_hi[cta] - alo, a.a_cap);
    // dose-limit constants of this CTA's rows, in the product arithmetic T
    T *arho = reinterpret_cast<T *>(smem + L.arho);
    T *acs = reinterpret_cast<T *>(smem + L.acs);
    T *aDl = reinterpret_cast<T *>(smem + L.aDl);
    T *aDu = reinterpret_cast<T *>(smem + L.aDu);
    uint8_t *afl = smem + L.afl;
    for (int i = tid; i < na; i += blockDim.x) {
      const int ai = alo + i;
      arho[i] = (T)a.P.rhoA[ai];
      acs[i] = (T)(a.cl[ai] + a.cu[ai]);
      aDl[i] = (T)a.Dl[ai];
      aDu[i] = (T)a.Du[ai];
      afl[i] = (uint8_t)((a.P.hasl[ai] ? 1 : 0) | (a.P.hasu[ai] ? 2 : 0));
    }
    __syncthreads();
    if (ps.nc > 0) {
      for (int s = 0; s < a.stages - 1; ++s) {
        if (a.producer == 0) issue_chunk_lsu(a, smem, L, ps);
        else if (tid == 0) issue_chunk(a, smem, L, ps);
        ps.seq_issue++;
      }
    }
  }

  // wait for every copy still in flight (bounded), so that the CTA never
  // exits with asynchronous writes into its shared memory pending
  static __device__ void drain(const PcgArgs &a, unsigned char *smem, PipeState &ps) {
    const CsrLayout L = lay(a);
    if (a.producer == 0) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      return;
    }
    bool ok = true;
    if (threadIdx.x == 0)
      for (uint32_t s = ps.seq_cons; s < ps.seq_issue; ++s) ok = wait(a, smem, L, s) && ok;
    if (!ok) atomicCAS(a.bar.err, 0, 7);
    __syncthreads();
  }


  // Row coefficient u_r = w2_r (P_r p) [+ rho (2 t (1/D_l + 1/D_u) + p_l - p_u)
  // for a dose-limit row; lane 0 writes its bottom entries and adds its share of
  // p'q to pqt].  All in the product arithmetic T.
  template <class T>
  static __device__ __forceinline__ T row_coef(const PcgArgs &a, const RowDesc &d, T dot,
                                               const double *ysrc, const double *pold,
                                               double beta, int alo, int na, const T *arho,
                                               const T *acs, const T *aDl, const T *aDu,
                                               const T *apl, const T *apu, const uint8_t *afl,
                                               int lane, T &pqt) {
    T u;
    // the row tables hold 2 sigma w of qp_create; wfac = sigma_now / sigma_create
    if constexpr (sizeof(T) == 4) u = (d.w2hi * a.P.wfac32) * dot;
    else u = (((double)d.w2hi + (double)d.w2lo) * a.P.wfac) * dot;
    if (d.a >= 0) {
      const DevProb &P = a.P;
      const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
      const int ai = d.a, il = ai - alo;
      T rho, cs, Dl, Du, pl, pu;
      int fl;
      if (il >= 0 && il < na) {
        rho = arho[il]; cs = acs[il]; Dl = aDl[il]; Du = aDu[il]; fl = afl[il];
        pl = apl[il]; pu = apu[il];
      } else {
        rho = (T)P.rhoA[ai]; cs = (T)(a.cl[ai] + a.cu[ai]); Dl = (T)a.Dl[ai]; Du = (T)a.Du[ai];
        fl = (P.hasl[ai] ? 1 : 0) | (P.hasu[ai] ? 2 : 0);
        pl = (T)((fl & 1) ? ldcg(ysrc + lo_off + ai) + beta * ldcg(pold + lo_off + ai) : 0.0);
        pu = (T)((fl & 2) ? ldcg(ysrc + up_off + ai) + beta * ldcg(pold + up_off + ai) : 0.0);
      }
      const T t = rho * dot;
      const T coef = (T)2 * t * cs + pl - pu;
      u += rho * coef;
      if (lane == 0) {
        const T ql = (fl & 1) ? t + Dl * pl : (T)0;
        const T qu = (fl & 2) ? -t + Du * pu : (T)0;
        a.qlam[P.me + ai] = (double)ql;
        a.qlam[P.me + P.m + ai] = (double)qu;
        pqt += pl * ql + pu * qu;
      }
    }
    return u;
  }

  // Rows of one staged chunk: dot with the p window, coefficient, scatter.
  // Returns this thread's share of p'(K p).  With T = float the per-row
  // coefficient is formed in FP32 (the FP64 pipe of the SM is narrow) and the
  // p'q partials are folded into FP64 once per chunk.
  template <class T, bool WIN>
  static __device__ double stage_rows(T &pqt, const PcgArgs &a, const double *ysrc, const double *pold,
                                      double beta, const float *sval, const int *scol,
                                      const RowDesc *sd, const T *pw, T *acc, T *accg, int lo,
                                      int alo, int na, const T *arho, const T *acs,
                                      const T *aDl, const T *aDu, const T *apl,
                                      const T *apu, const uint8_t *afl, double *s_bcast) {
    const DevProb &P = a.P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
    double pq = 0.0;
    const int nrows = sd[0].off;
    if (WIN && sd[0].a < 0 && sd[0].w2hi != 0.f) {
      // two rows per warp, at most 128 nonzeros each: fixed-trip loops, values
      // and columns kept in registers between the dot and the scatter
      for (int i = 2 * warp; i < nrows; i += 2 * nw) {
        const bool two = i + 1 < nrows;
        const RowDesc d0 = sd[1 + i];
        const int e0 = sd[2 + i].off;
        const RowDesc d1 = two ? sd[2 + i] : d0;
        const int e1 = two ? sd[3 + i].off : d0.off;
        float v0[4], v1[4];
        int c0[4], c1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k0 = d0.off + lane + 32 * q, k1 = d1.off + lane + 32 * q;
          const bool ok0 = k0 < e0, ok1 = k1 < e1;
          c0[q] = ok0 ? scol[k0] - lo : -1;
          v0[q] = ok0 ? sval[k0] : 0.f;
          c1[q] = ok1 ? scol[k1] - lo : -1;
          v1[q] = ok1 ? sval[k1] : 0.f;
        }
        T s0 = (T)0, s1 = (T)0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (c0[q] >= 0) s0 += (T)v0[q] * pw[c0[q]];
          if (c1[q] >= 0) s1 += (T)v1[q] * pw[c1[q]];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        const T u0 = row_coef<T>(a, d0, s0, ysrc, pold, beta, alo, na, arho, acs, aDl, aDu, apl,
                                 apu, afl, lane, pqt);
        const T u1 = two ? row_coef<T>(a, d1, s1, ysrc, pold, beta, alo, na, arho, acs, aDl, aDu,
                                       apl, apu, afl, lane, pqt)
                         : (T)0;
        if (lane == 0) pqt += u0 * s0 + u1 * s1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (c0[q] >= 0) atomicAdd(acc + c0[q], u0 * (T)v0[q]);
          if (c1[q] >= 0) atomicAdd(acc + c1[q], u1 * (T)v1[q]);
        }
      }
    } else if (sd[0].a < 0) {
      for (int i = warp; i < nrows; i += nw) {
        const RowDesc d = sd[1 + i];
        const int end = sd[2 + i].off;
        T dot = (T)0;
        for (int k = d.off + lane; k < end; k += 32) {
          const int c = scol[k];
          T pv;
          if constexpr (WIN) pv = pw[c - lo];
          else pv = (T)(ldcg(ysrc + c) + beta * ldcg(pold + c));
          dot += (T)sval[k] * pv;
        }
        dot = warp_sum(dot);
        const T u = row_coef<T>(a, d, dot, ysrc, pold, beta, alo, na, arho, acs, aDl, aDu, apl,
                                apu, afl, lane, pqt);
        if (lane == 0) pqt += u * dot;
        for (int k = d.off + lane; k < end; k += 32) {
          const int c = scol[k];
          if constexpr (WIN) atomicAdd(acc + (c - lo), u * (T)sval[k]);
          else atomicAdd(accg + c, u * (T)sval[k]);
        }
      }
    } else {
      // a single row longer than a stage: whole CTA, straight from global memory
      const int64_t r = sd[0].a;
      const RowDesc d = sd[1];
      const int64_t s = P.rowptr[r], e = P.rowptr[r + 1];
      double part[1] = {0.0};
      for (int64_t k = s + tid; k < e; k += blockDim.x) {
        const int c = P.col[k];
        T pv;
        if constexpr (WIN) pv = pw[c - lo];
        else pv = (T)(ldcg(ysrc + c) + beta * ldcg(pold + c));
        part[0] += (double)((T)P.val[k] * pv);
      }
      __shared__ double shl[32];
      block_sum<1>(part, shl);
      if (tid == 0) {
        const double dd = part[0];
        double ud = ((double)d.w2hi + (double)d.w2lo) * P.wfac * dd;
        if (d.a >= 0) {
          const int ai = d.a;
          const double rho = P.rhoA[ai];
          const int fl = (P.hasl[ai] ? 1 : 0) | (P.hasu[ai] ? 2 : 0);
          const double pl = (fl & 1) ? ldcg(ysrc + lo_off + ai) + beta * ldcg(pold + lo_off + ai) : 0.0;
          const double pu = (fl & 2) ? ldcg(ysrc + up_off + ai) + beta * ldcg(pold + up_off + ai) : 0.0;
          const double t = rho * dd;
          const double coef = 2.0 * t * (a.cl[ai] + a.cu[ai]) + pl - pu;
          ud += rho * coef;
          const double ql = (fl & 1) ? t + a.Dl[ai] * pl : 0.0;
          const double qu = (fl & 2) ? -t + a.Du[ai] * pu : 0.0;
          a.qlam[P.me + ai] = ql;
          a.qlam[P.me + P.m + ai] = qu;
          pq += pl * ql + pu * qu;
        }
        pq += ud * dd;
        s_bcast[0] = ud;
      }
      __syncthreads();
      const T u = (T)s_bcast[0];
      for (int64_t k = s + tid; k < e; k += blockDim.x) {
        const int c = P.col[k];
        if constexpr (WIN) atomicAdd(acc + (c - lo), u * (T)P.val[k]);
        else atomicAdd(accg + c, u * (T)P.val[k]);
      }
    }
    return pq;
  }

  template <class T>
  static __device__ double phaseA(const PcgArgs &a, const double *ysrc, const double *pold,
                                  double *pnew, double beta, int64_t vb, int64_t ve,
                                  unsigned char *smem, PipeState &ps, bool &ok) {
    const DevProb &P = a.P;
    const CsrLayout L = lay(a);
    const int cta = blockIdx.x, tid = threadIdx.x;
    const int lo = a.win_lo[cta], hi = a.win_hi[cta];
    const int wlen = hi - lo;
    const bool win = wlen <= a.win_cap;
    T *pw = reinterpret_cast<T *>(smem + L.pw);
    T *acc = reinterpret_cast<T *>(smem + L.acc);
    T *accg = reinterpret_cast<T *>(a.accx);
    const int alo = a.a_lo[cta], na = min(a.a_hi[cta] - alo, a.a_cap);
    const T *arho = reinterpret_cast<const T *>(smem + L.arho);
    const T *acs = reinterpret_cast<const T *>(smem + L.acs);
    const T *aDl = reinterpret_cast<const T *>(smem + L.aDl);
    const T *aDu = reinterpret_cast<const T *>(smem + L.aDu);
    T *apl = reinterpret_cast<T *>(smem + L.apl);
    T *apu = reinterpret_cast<T *>(smem + L.apu);
    const uint8_t *afl = smem + L.afl;
    const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
    double pq = write_owned_p(a, ysrc, pold, pnew, beta, vb, ve);
    if (win) {
      for (int j = tid; j < wlen; j += blockDim.x) {
        const int c = lo + j;
        pw[j] = (T)(ldcg(ysrc + c) + beta * ldcg(pold + c));
        acc[j] = (T)0;
      }
    }
    for (int i = tid; i < na; i += blockDim.x) {
      const int ai = alo + i;
      apl[i] = (T)((afl[i] & 1) ? ldcg(ysrc + lo_off + ai) + beta * ldcg(pold + lo_off + ai) : 0.0);
      apu[i] = (T)((afl[i] & 2) ? ldcg(ysrc + up_off + ai) + beta * ldcg(pold + up_off + ai) : 0.0);
    }
    __syncthreads();
    __shared__ double s_bcast[2];
    T pqt = (T)0;   // FP32 (mixed) share of p'q, folded into FP64 once per product
    for (int j = 0; j < ps.nc; ++j) {
      if (a.producer == 0) {
        issue_chunk_lsu(a, smem, L, ps);
        ps.seq_issue++;
        cp_async_wait_pending(a.stages - 1);    // the group of seq_cons has landed
        __syncthreads();
      } else {
      if (tid == 0) issue_chunk(a, smem, L, ps);
      ps.seq_issue++;
      // one thread waits (bounded); the others park on the CTA barrier instead
      // of polling the mbarrier in shared memory, then take the (already
      // completed) phase with one non-blocking test for acquire ordering
      bool w = true;
      if (tid == 0) w = wait(a, smem, L, ps.seq_cons);
      if (__syncthreads_or(!w)) {
        if (tid == 0) atomicCAS(a.bar.err, 0, 7);
        ok = false;
        return 0.0;
      }
      if (tid != 0)
        (void)mbar_try_wait(reinterpret_cast<uint64_t *>(smem + L.bar) + (ps.seq_cons % (uint32_t)a.stages),
                            (ps.seq_cons / (uint32_t)a.stages) & 1u);
      }
      const int st = (int)(ps.seq_cons % (uint32_t)a.stages);
      const unsigned char *sb = smem + L.stage0 + (size_t)st * L.stage_bytes;
      const float *sval = reinterpret_cast<const float *>(sb + L.val_off);
      const int *scol = reinterpret_cast<const int *>(sb + L.col_off);
      const RowDesc *sd = reinterpret_cast<const RowDesc *>(sb + L.desc_off);
      if (win)
        pq += stage_rows<T, true>(pqt, a, ysrc, pold, beta, sval, scol, sd, pw, acc, accg, lo, alo,
                                  na, arho, acs, aDl, aDu, apl, apu, afl, s_bcast);
      else
        pq += stage_rows<T, false>(pqt, a, ysrc, pold, beta, sval, scol, sd, pw, acc, accg, lo, alo,
                                   na, arho, acs, aDl, aDu, apl, apu, afl, s_bcast);
      __syncthreads();
      ps.seq_cons++;
    }
    pq += (double)pqt;
    if (win) {
      for (int j = tid; j < wlen; j += blockDim.x) {
        const T v = acc[j];
        if (v != (T)0) atomicAdd(accg + lo + j, v);
      }
    }
    return pq;
  }
};

// ---------------------------------------------------------------- CSR, register-streamed
// Shared memory of the register-streamed operator: the p window, one private
// accumulator per warp (no atomics in the scatter), the dose-limit constants.
struct RowsLayout { size_t pw, acc, arho, acs, aDl, aDu, apl, apu, afl, total; };
// es = size of the product type (4: FP32 products, 8: FP64 products)
__host__ __device__ inline RowsLayout rows_layout(int rws, int nw, int a_cap, int es) {
  RowsLayout L;
  size_t o = 0;
  L.pw = o; o += es * (size_t)rws;
  L.acc = o; o += es * (size_t)rws * nw;
  L.arho = o; o += es * (size_t)a_cap;
  L.acs = o; o += es * (size_t)a_cap;
  L.aDl = o; o += es * (size_t)a_cap;
  L.aDu = o; o += es * (size_t)a_cap;
  L.apl = o; o += es * (size_t)a_cap;
  L.apu = o; o += es * (size_t)a_cap;
  L.afl = o; o += (size_t)a_cap;
  L.total = kq_up128(o);
  return L;
}

// L2 bulk prefetch; the caller passes a 16-byte aligned address
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  if (bytes >= 16)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes & ~15u) : "memory");
}

// Every warp walks its own rows (pairs 2w, 2w+1, then +2 NW, ...) with plain
// 16-byte loads straight into registers, two pairs' loads in flight while the
// current pair is processed (optionally, KQ_PF > 0, thread 0 also prefetches
// the CTA's rows into L2; measured slower on the dose QP, so off by default).
// No shared-memory staging and no CTA barrier inside the product.  The scatter goes into the warp's private accumulator
// with plain read-modify-write: the columns of one row are distinct (padding
// included), and __syncwarp orders the rows of a warp.  The private copies
// are summed once per product.
struct OpCsrRows {
  // The CTA's rows occupy the contiguous lane-group range [base, end); the L2
  // prefetch cuts it into one piece per warp step (no loads needed to find it).
  static __device__ __forceinline__ int *pf_state() {
    __shared__ int s_pf[3];   // base, end, groups per step
    return s_pf;
  }
  // thread 0: L2 prefetch of the piece of warp step `step`
  static __device__ __forceinline__ void prefetch_step(const PcgArgs &a, int step) {
    const int *st = pf_state();
    const int b = st[0] + step * st[2], e = min(st[1], b + st[2]);
    if (b >= e) return;
    // values: float4 groups, 16-byte aligned
    prefetch_l2(a.rval4 + b, (uint32_t)(e - b) * 16u);
    // columns: 8 bytes per group; the bulk prefetch needs a 16-byte aligned
    // start and size, so the byte range is rounded out to 16-byte boundaries
    // (the column array ends with one spare group, so the end stays inside it)
    const uint64_t cb = ((uint64_t)b * 8u) & ~(uint64_t)15;
    const uint64_t ce = ((uint64_t)e * 8u + 15u) & ~(uint64_t)15;
    prefetch_l2(reinterpret_cast<const unsigned char *>(a.rcol2) + cb, (uint32_t)(ce - cb));
  }

  template <class T>
  static __device__ void begin(const PcgArgs &a, unsigned char *smem) {
    const int cta = blockIdx.x, tid = threadIdx.x, nw = blockDim.x >> 5;
    const RowsLayout L = rows_layout(a.rws, nw, a.a_cap, (int)sizeof(T));
    T *acc = reinterpret_cast<T *>(smem + L.acc);
    for (int j = tid; j < a.rws * nw; j += blockDim.x) acc[j] = (T)0;
    const int alo = a.a_lo[cta], na = min(a.a_hi[cta] - alo, a.a_cap);
    T *arho = reinterpret_cast<T *>(smem + L.arho);
    T *acs = reinterpret_cast<T *>(smem + L.acs);
    T *aDl = reinterpret_cast<T *>(smem + L.aDl);
    T *aDu = reinterpret_cast<T *>(smem + L.aDu);
    uint8_t *afl = smem + L.afl;
    for (int i = tid; i < na; i += blockDim.x) {
      const int ai = alo + i;
      arho[i] = (T)a.P.rhoA[ai];
      acs[i] = (T)(a.cl[ai] + a.cu[ai]);
      aDl[i] = (T)a.Dl[ai];
      aDu[i] = (T)a.Du[ai];
      afl[i] = (uint8_t)((a.P.hasl[ai] ? 1 : 0) | (a.P.hasu[ai] ? 2 : 0));
    }
    if (tid == 0) {
      const int64_t r0 = a.row_begin[cta];
      const int nr = (int)(a.row_begin[cta + 1] - r0);
      int *st = pf_state();
      st[0] = st[1] = st[2] = 0;
      if (nr > 0) {
        const RowSlot f = a.rslot[r0], l = a.rslot[r0 + nr - 1];
        const int nsteps = (nr + 2 * nw - 1) / (2 * nw);
        st[0] = f.off4;
        st[1] = l.off4 + l.len4;
        st[2] = (st[1] - st[0] + nsteps - 1) / nsteps;
      }
      if (a.pf_dist > 0)
        for (int s = 0; s < a.pf_dist; ++s) prefetch_step(a, s);
    }
    __syncthreads();
  }

  // FP64 products in double-float: one row's scatter of u P_r into the warp's
  // accumulator held as float pairs (columns distinct)
  static __device__ __forceinline__ void scatter_df(float2 *accw, const float4 &v, const int4 &c,
                                                    double u, bool act) {
    if (act) {
      float uh, ul;
      df_split(u, uh, ul);
      const float2 a0 = accw[c.x], a1 = accw[c.y], a2 = accw[c.z], a3 = accw[c.w];
      DFAcc t0{a0.x, a0.y}, t1{a1.x, a1.y}, t2{a2.x, a2.y}, t3{a3.x, a3.y};
      t0.add_prod(v.x, uh, ul);
      t1.add_prod(v.y, uh, ul);
      t2.add_prod(v.z, uh, ul);
      t3.add_prod(v.w, uh, ul);
      accw[c.x] = make_float2(t0.h, t0.l);
      accw[c.y] = make_float2(t1.h, t1.l);
      accw[c.z] = make_float2(t2.h, t2.l);
      accw[c.w] = make_float2(t3.h, t3.l);
    }
    __syncwarp();
  }

  // one row's scatter into the warp's accumulator (columns distinct)
  template <class T>
  static __device__ __forceinline__ void scatter(T *accw, const T (&v)[4], const int4 &c, T u,
                                                 bool act) {
    if (act) {
      const T a0 = accw[c.x], a1 = accw[c.y], a2 = accw[c.z], a3 = accw[c.w];
      accw[c.x] = a0 + u * v[0];
      accw[c.y] = a1 + u * v[1];
      accw[c.z] = a2 + u * v[2];
      accw[c.w] = a3 + u * v[3];
    }
    __syncwarp();
  }

  template <class T>
  static __device__ double phaseA(const PcgArgs &a, const double *ysrc, const double *pold,
                                  double *pnew, double beta, int64_t vb, int64_t ve,
                                  unsigned char *smem, bool &ok) {
    const DevProb &P = a.P;
    const int cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    const RowsLayout L = rows_layout(a.rws, nw, a.a_cap, (int)sizeof(T));
    const int lo = a.win_lo[cta], wlen = a.win_hi[cta] - lo;
    T *pw = reinterpret_cast<T *>(smem + L.pw);
    T *acc = reinterpret_cast<T *>(smem + L.acc);
    T *accw = acc + (size_t)warp * a.rws;
    T *accg = reinterpret_cast<T *>(a.accx);
    const int alo = a.a_lo[cta], na = min(a.a_hi[cta] - alo, a.a_cap);
    const T *arho = reinterpret_cast<const T *>(smem + L.arho);
    const T *acs = reinterpret_cast<const T *>(smem + L.acs);
    const T *aDl = reinterpret_cast<const T *>(smem + L.aDl);
    const T *aDu = reinterpret_cast<const T *>(smem + L.aDu);
    T *apl = reinterpret_cast<T *>(smem + L.apl);
    T *apu = reinterpret_cast<T *>(smem + L.apu);
    const uint8_t *afl = smem + L.afl;
    const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
    const int64_t r0 = a.row_begin[cta];
    const int nr = (int)(a.row_begin[cta + 1] - r0);
    const RowSlot *S = a.rslot + r0;
    // Loads run ahead of the arithmetic: slot descriptors three pair-steps
    // ahead, values and columns two; the first steps do not depend on p and
    // start before the window is filled.
    auto ld_slots = [&](int ii, RowSlot &x0, RowSlot &x1) {
      x0 = RowSlot{0, 0, -1, 0.f};
      x1 = RowSlot{0, 0, -1, 0.f};
      if (ii < nr) x0 = S[ii];
      if (ii + 1 < nr) x1 = S[ii + 1];
    };
    auto ld_data = [&](const RowSlot &x0, const RowSlot &x1, float4 &v0, float4 &v1, uint2 &c0,
                       uint2 &c1) {
      v0 = make_float4(0.f, 0.f, 0.f, 0.f);
      v1 = v0;
      c0 = make_uint2(0u, 0u);
      c1 = c0;
      if (lane < x0.len4) { v0 = __ldcs(a.rval4 + x0.off4 + lane); c0 = __ldcs(a.rcol2 + x0.off4 + lane); }
      if (lane < x1.len4) { v1 = __ldcs(a.rval4 + x1.off4 + lane); c1 = __ldcs(a.rcol2 + x1.off4 + lane); }
    };
    T pqt = (T)0;
    // one pair of rows: dots with the window, coefficients, scatter (FP32
    // products; FP64 products take process_df below)
    auto process = [&](int ii, const RowSlot &s0, const RowSlot &s1, const float4 &v0,
                       const float4 &v1, const uint2 &p0, const uint2 &p1) {
      const int4 c0 = make_int4((int)(p0.x & 0xffffu), (int)(p0.x >> 16), (int)(p0.y & 0xffffu),
                                (int)(p0.y >> 16));
      const int4 c1 = make_int4((int)(p1.x & 0xffffu), (int)(p1.x >> 16), (int)(p1.y & 0xffffu),
                                (int)(p1.y >> 16));
      const bool has1 = ii + 1 < nr;
      const bool act0 = lane < s0.len4, act1 = lane < s1.len4;
      const float w0lo = 0.f, w1lo = 0.f;
      const T x0[4] = {(T)v0.x, (T)v0.y, (T)v0.z, (T)v0.w};
      const T x1[4] = {(T)v1.x, (T)v1.y, (T)v1.z, (T)v1.w};
      T d0 = (T)0, d1 = (T)0;
      if (act0) d0 = x0[0] * pw[c0.x] + x0[1] * pw[c0.y] + x0[2] * pw[c0.z] + x0[3] * pw[c0.w];
      if (act1) d1 = x1[0] * pw[c1.x] + x1[1] * pw[c1.y] + x1[2] * pw[c1.z] + x1[3] * pw[c1.w];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      }
      const RowDesc rd0{0, s0.a, s0.w2, w0lo}, rd1{0, s1.a, s1.w2, w1lo};
      const T u0 = OpCsrStaged::row_coef<T>(a, rd0, d0, ysrc, pold, beta, alo, na, arho, acs, aDl,
                                            aDu, apl, apu, afl, lane, pqt);
      T u1 = (T)0;
      if (has1)
        u1 = OpCsrStaged::row_coef<T>(a, rd1, d1, ysrc, pold, beta, alo, na, arho, acs, aDl, aDu,
                                      apl, apu, afl, lane, pqt);
      if (lane == 0) pqt += u0 * d0 + u1 * d1;
      scatter<T>(accw, x0, c0, u0, act0);
      scatter<T>(accw, x1, c1, u1, act1);
    };
    // FP64 products in double-float (window and accumulators as float pairs,
    // the FP32 matrix values exact): dots, coefficients in FP64, scatter
    auto process_df = [&](int ii, const RowSlot &s0, const RowSlot &s1, const float4 &v0,
                          const float4 &v1, const uint2 &p0, const uint2 &p1) {
      const float2 *pw2 = reinterpret_cast<const float2 *>(pw);
      float2 *acc2w = reinterpret_cast<float2 *>(accw);
      const int4 c0 = make_int4((int)(p0.x & 0xffffu), (int)(p0.x >> 16), (int)(p0.y & 0xffffu),
                                (int)(p0.y >> 16));
      const int4 c1 = make_int4((int)(p1.x & 0xffffu), (int)(p1.x >> 16), (int)(p1.y & 0xffffu),
                                (int)(p1.y >> 16));
      const bool has1 = ii + 1 < nr;
      const bool act0 = lane < s0.len4, act1 = lane < s1.len4;
      const float w0lo = __ldg(a.rw2lo + r0 + ii), w1lo = has1 ? __ldg(a.rw2lo + r0 + ii + 1) : 0.f;
      DFAcc q0, q1;
      if (act0) {
        const float2 g0 = pw2[c0.x], g1 = pw2[c0.y], g2 = pw2[c0.z], g3 = pw2[c0.w];
        q0.add_prod(v0.x, g0.x, g0.y);
        q0.add_prod(v0.y, g1.x, g1.y);
        q0.add_prod(v0.z, g2.x, g2.y);
        q0.add_prod(v0.w, g3.x, g3.y);
      }
      if (act1) {
        const float2 g0 = pw2[c1.x], g1 = pw2[c1.y], g2 = pw2[c1.z], g3 = pw2[c1.w];
        q1.add_prod(v1.x, g0.x, g0.y);
        q1.add_prod(v1.y, g1.x, g1.y);
        q1.add_prod(v1.z, g2.x, g2.y);
        q1.add_prod(v1.w, g3.x, g3.y);
      }
      q0.warp_reduce();
      q1.warp_reduce();
      const T d0 = (T)q0.value(), d1 = (T)q1.value();
      const RowDesc rd0{0, s0.a, s0.w2, w0lo}, rd1{0, s1.a, s1.w2, w1lo};
      const T u0 = OpCsrStaged::row_coef<T>(a, rd0, d0, ysrc, pold, beta, alo, na, arho, acs, aDl,
                                            aDu, apl, apu, afl, lane, pqt);
      T u1 = (T)0;
      if (has1)
        u1 = OpCsrStaged::row_coef<T>(a, rd1, d1, ysrc, pold, beta, alo, na, arho, acs, aDl, aDu,
                                      apl, apu, afl, lane, pqt);
      if (lane == 0) pqt += u0 * d0 + u1 * d1;
      scatter_df(acc2w, v0, c0, (double)u0, act0);
      scatter_df(acc2w, v1, c1, (double)u1, act1);
    };
    int i = 2 * warp;
    const int stp = 2 * nw;
    RowSlot sa0, sa1, sb0, sb1, sc0, sc1;
    float4 va0, va1, vb0, vb1;
    uint2 ca0, ca1, cb0, cb1;
    ld_slots(i, sa0, sa1);
    ld_slots(i + stp, sb0, sb1);
    ld_slots(i + 2 * stp, sc0, sc1);
    double pq = 0.0;
    const float *p32o = (a.apply || sizeof(T) != 4) ? nullptr : p32_of(a, pold);
    constexpr int KW = 6;
    if (p32o && a.y32 && wlen + 2 * na <= KW * (int)blockDim.x) {
      // window p from the FP32 copies of y and p_old (FP32 arithmetic: the
      // product rounds p to FP32 anyway).  One index space: window columns,
      // then the A rows' lower and upper entries.  The window loads are issued
      // before the owned-entry update, so both take one memory round trip.
      const float b32 = (float)beta;
      const int tot = wlen + 2 * na;
      float yv[KW], pv[KW];
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int j = tid + k * (int)blockDim.x;
        yv[k] = 0.f;
        pv[k] = 0.f;
        if (j < tot) {
          bool need = true;
          int64_t ix;
          if (j < wlen) {
            ix = lo + j;
          } else {
            const int q = (j - wlen) >> 1, up = (j - wlen) & 1;
            ix = (up ? up_off : lo_off) + alo + q;
            need = (afl[q] & (up ? 2 : 1)) != 0;
          }
          if (need) {
            yv[k] = __ldcg(a.y32 + ix);
            pv[k] = __ldcg(p32o + ix);
          }
        }
      }
      ld_data(sa0, sa1, va0, va1, ca0, ca1);
      ld_data(sb0, sb1, vb0, vb1, cb0, cb1);
      pq = write_owned_p(a, ysrc, pold, pnew, beta, vb, ve);
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int j = tid + k * (int)blockDim.x;
        if (j < tot) {
          const T v = (T)fmaf(b32, pv[k], yv[k]);
          if (j < wlen) {
            pw[j] = v;
          } else {
            const int q = (j - wlen) >> 1;
            if ((j - wlen) & 1) apu[q] = v; else apl[q] = v;
          }
        }
      }
    } else if (p32o && a.y32) {
      pq = write_owned_p(a, ysrc, pold, pnew, beta, vb, ve);
      ld_data(sa0, sa1, va0, va1, ca0, ca1);
      ld_data(sb0, sb1, vb0, vb1, cb0, cb1);
      const float b32 = (float)beta;
      for (int j = tid; j < wlen + 2 * na; j += blockDim.x) {
        if (j < wlen) {
          const int c = lo + j;
          pw[j] = (T)fmaf(b32, __ldcg(p32o + c), __ldcg(a.y32 + c));
        } else {
          const int k = (j - wlen) >> 1, up = (j - wlen) & 1;
          const int64_t ix = (up ? up_off : lo_off) + alo + k;
          const float v = (afl[k] & (up ? 2 : 1)) ? fmaf(b32, __ldcg(p32o + ix), __ldcg(a.y32 + ix)) : 0.f;
          if (up) apu[k] = (T)v; else apl[k] = (T)v;
        }
      }
    } else {
      pq = write_owned_p(a, ysrc, pold, pnew, beta, vb, ve);
      ld_data(sa0, sa1, va0, va1, ca0, ca1);
      ld_data(sb0, sb1, vb0, vb1, cb0, cb1);
      for (int j = tid; j < wlen; j += blockDim.x) {
        const int c = lo + j;
        const double v = ldcg(ysrc + c) + beta * ldcg(pold + c);
        if constexpr (sizeof(T) == 8) {
          float h, l;
          df_split(v, h, l);
          reinterpret_cast<float2 *>(pw)[j] = make_float2(h, l);
        } else {
          pw[j] = (T)v;
        }
      }
      for (int k = tid; k < na; k += blockDim.x) {
        const int ai = alo + k;
        apl[k] = (T)((afl[k] & 1) ? ldcg(ysrc + lo_off + ai) + beta * ldcg(pold + lo_off + ai) : 0.0);
        apu[k] = (T)((afl[k] & 2) ? ldcg(ysrc + up_off + ai) + beta * ldcg(pold + up_off + ai) : 0.0);
      }
    }
    __syncthreads();
    int step = 0;
    for (; i < nr; i += stp, ++step) {
      if (tid == 0 && a.pf_dist > 0) prefetch_step(a, step + a.pf_dist);
      RowSlot sd0, sd1;
      float4 vc0, vc1;
      uint2 cc0, cc1;
      ld_slots(i + 3 * stp, sd0, sd1);
      ld_data(sc0, sc1, vc0, vc1, cc0, cc1);
      if constexpr (sizeof(T) == 8) process_df(i, sa0, sa1, va0, va1, ca0, ca1);
      else process(i, sa0, sa1, va0, va1, ca0, ca1);
      sa0 = sb0; sa1 = sb1; sb0 = sc0; sb1 = sc1; sc0 = sd0; sc1 = sd1;
      va0 = vb0; va1 = vb1; ca0 = cb0; ca1 = cb1;
      vb0 = vc0; vb1 = vc1; cb0 = cc0; cb1 = cc1;
    }
    __syncthreads();
    // sum the private copies into the global accumulator; zero them
    if constexpr (sizeof(T) == 8) {
      // the private copies hold float pairs (two columns per 16 bytes)
      float4 *accp = reinterpret_cast<float4 *>(acc);
      const int ws2 = a.rws >> 1;
      for (int j2 = tid; j2 < ws2; j2 += blockDim.x) {
        DFAcc t0, t1;
        for (int w = 0; w < nw; ++w) {
          const float4 x = accp[(size_t)w * ws2 + j2];
          t0.add(x.x, x.y);
          t1.add(x.z, x.w);
          accp[(size_t)w * ws2 + j2] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const double tx = t0.value(), ty = t1.value();
        const int c = 2 * j2;
        if (c < wlen && tx != 0.0) atomicAdd(reinterpret_cast<double *>(accg) + lo + c, tx);
        if (c + 1 < wlen && ty != 0.0) atomicAdd(reinterpret_cast<double *>(accg) + lo + c + 1, ty);
      }
      (void)ok;
      return pq + (double)pqt;
    }
    float4 *acc4 = reinterpret_cast<float4 *>(reinterpret_cast<float *>(acc));
    const int ws4 = a.rws >> 2;
    for (int j4 = tid; j4 < ws4; j4 += blockDim.x) {
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int w = 0; w < nw; ++w) {
        const float4 x = acc4[(size_t)w * ws4 + j4];
        t.x += x.x; t.y += x.y; t.z += x.z; t.w += x.w;
        acc4[(size_t)w * ws4 + j4] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const int c = 4 * j4;
      if (c + 3 < wlen) {
        // lo is a multiple of 4: one 16-byte vector reduction
        if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f)
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(reinterpret_cast<float *>(accg) + lo + c),
                       "f"(t.x), "f"(t.y), "f"(t.z), "f"(t.w) : "memory");
      } else {
        float *ag = reinterpret_cast<float *>(accg);
        if (c + 0 < wlen && t.x != 0.f) atomicAdd(ag + lo + c + 0, t.x);
        if (c + 1 < wlen && t.y != 0.f) atomicAdd(ag + lo + c + 1, t.y);
        if (c + 2 < wlen && t.z != 0.f) atomicAdd(ag + lo + c + 2, t.z);
      }
    }
    // prefetch the first steps of the next product (the matrix does not change)
    if (tid == 0 && a.pf_dist > 0)
      for (int s2 = 0; s2 < a.pf_dist; ++s2) prefetch_step(a, s2);
    (void)ok;
    return pq + (double)pqt;
  }
};

template <class OP> struct IsStaged { static constexpr bool value = false; };
template <> struct IsStaged<OpCsrStaged> { static constexpr bool value = true; };

template <class OP> struct IsRows { static constexpr bool value = false; };
template <> struct IsRows<OpCsrRows> { static constexpr bool value = true; };

template <class OP> struct IsLowrank { static constexpr bool value = false; };
template <class ZS> struct IsLowrank<OpLowrank<ZS>> { static constexpr bool value = true; };

// ---------------------------------------------------------------- general rows of a CSR A (any operator)
// Rows of a CSR A, and (for the CSR least-squares operators, whose passes
// read only P) the dense equality rows C, one warp per row over the warps of
// the problem's CTAs: t = rho A_i p_x, coefficient 2 t (1/D_l + 1/D_u) + p_l -
// p_u scattered into the top block with global atomics (the columns of a
// general row can be anywhere in [0, n)), bottom entries (t + D_l p_l,
// -t + D_u p_u) written directly.  Returns this thread's share of p'Kp.
template <class T, class AS>
__device__ double csr_a_rows(const PcgArgs &a, const double *ysrc, const double *pold, double beta,
                             int vcta, int vG) {
  const DevProb &P = a.P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t n = P.n, m = P.m, me = P.me;
  const int64_t lo_off = n + me, up_off = n + me + m;
  const int64_t gw0 = (int64_t)vcta * nw + warp, GW = (int64_t)vG * nw;
  T *accg = reinterpret_cast<T *>(a.accx);
  const AS *val = reinterpret_cast<const AS *>(P.aval);
  double pq = 0.0;
  if (P.akind == KQ_A_CSR) {
    for (int64_t ai = gw0; ai < m; ai += GW) {
      const bool hl = P.hasl[ai] != 0, hu = P.hasu[ai] != 0;
      if (!hl && !hu) {
        if (lane == 0) { a.qlam[me + ai] = 0.0; a.qlam[me + m + ai] = 0.0; }
        continue;
      }
      const int64_t k0 = P.arowptr[ai], k1 = P.arowptr[ai + 1];
      T dot = (T)0;
      for (int64_t k = k0 + lane; k < k1; k += 32) {
        const int c = P.acol[k];
        dot += (T)ld_as_f64(val, k) * (T)(ldcg(ysrc + c) + beta * ldcg(pold + c));
      }
      dot = warp_sum(dot);
      const double rho_a = P.rhoA[ai];
      const double t = rho_a * (double)dot;
      const double pl = hl ? ldcg(ysrc + lo_off + ai) + beta * ldcg(pold + lo_off + ai) : 0.0;
      const double pu = hu ? ldcg(ysrc + up_off + ai) + beta * ldcg(pold + up_off + ai) : 0.0;
      const double coef = 2.0 * t * (a.cl[ai] + a.cu[ai]) + pl - pu;
      const T cf = (T)(coef * rho_a);
      for (int64_t k = k0 + lane; k < k1; k += 32) atomicAdd(accg + P.acol[k], cf * (T)ld_as_f64(val, k));
      if (lane == 0) {
        const double ql = hl ? t + a.Dl[ai] * pl : 0.0;
        const double qu = hu ? -t + a.Du[ai] * pu : 0.0;
        a.qlam[me + ai] = ql;
        a.qlam[me + m + ai] = qu;
        pq += coef * t + pl * ql + pu * qu;
      }
    }
  }
  if (P.hkind == KQ_H_CSR_LSQ) {
    // equality rows (scaled, dense): t = C_e p_x, coefficient 2 t / mu + p_e
    for (int64_t e = gw0; e < me; e += GW) {
      const double *cr = P.Cd + e * n;
      T dot = (T)0;
      for (int64_t j = lane; j < n; j += 32) dot += (T)cr[j] * (T)(ldcg(ysrc + j) + beta * ldcg(pold + j));
      dot = warp_sum(dot);
      const double t = (double)dot;
      const double pe = ldcg(ysrc + n + e) + beta * ldcg(pold + n + e);
      const double coef = 2.0 * t / mu_of(a) + pe;
      const T cf = (T)coef;
      for (int64_t j = lane; j < n; j += 32) {
        const T v = cf * (T)cr[j];
        if (v != (T)0) atomicAdd(accg + j, v);
      }
      if (lane == 0) {
        const double qe = t + mu_of(a) * pe;
        a.qlam[e] = qe;
        pq += coef * t + pe * qe;
      }
    }
  }
  return pq;
}

template <class T>
__device__ __forceinline__ double extra_rows(const PcgArgs &a, const double *ysrc, const double *pold,
                                             double beta, int vcta, int vG) {
  if (a.P.akind != KQ_A_CSR && !(a.P.hkind == KQ_H_CSR_LSQ && a.P.me > 0)) return 0.0;
  if (a.P.adtype == KQ_F32) return csr_a_rows<T, float>(a, ysrc, pold, beta, vcta, vG);
  return csr_a_rows<T, double>(a, ysrc, pold, beta, vcta, vG);
}

template <class OP, class T>
__device__ __forceinline__ double run_phaseA(const PcgArgs &a, const double *ysrc,
                                             const double *pold, double *pnew, double beta,
                                             int64_t vb, int64_t ve, unsigned char *smem,
                                             PipeState &ps, bool &ok, int vcta, int vG) {
  double pq;
  ok = true;
  if constexpr (IsLowrank<OP>::value || IsRows<OP>::value) {
    pq = OP::template phaseA<T>(a, ysrc, pold, pnew, beta, vb, ve, smem, ok);
  } else if constexpr (IsStaged<OP>::value) {
    pq = OP::template phaseA<T>(a, ysrc, pold, pnew, beta, vb, ve, smem, ps, ok);
  } else {
    pq = OP::template phaseA<T>(a, ysrc, pold, pnew, beta, vb, ve, smem, vcta, vG, ok);
  }
  if (ok) pq += extra_rows<T>(a, ysrc, pold, beta, vcta, vG);
  return pq;
}

// The PCG solve (or one product in APPLY mode) of one problem by the CTAs
// cta = 0..G-1 (the whole grid, or one team of the batched solver).
// Sum of G slot values by warp 0 in a fixed order, the loads of up to 160
// slots issued together (one memory round trip).
__device__ __forceinline__ double slot_sum_w0(const double *s, int G) {
  double v = 0.0;
  for (int b = 0; b < G; b += 160) {
    double t[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int i = b + threadIdx.x + 32 * k;
      t[k] = (i < G) ? __ldcg(s + i) : 0.0;
    }
    v += ((t[0] + t[1]) + (t[2] + t[3])) + t[4];
  }
  return warp_sum(v);
}

// Sum of two slot arrays by warp 0 (the fixed order of slot_sum_w0); both
// arrays' loads are issued before any arithmetic, so the two sums cost one
// memory round trip after the grid barrier instead of two.  Result in warp 0.
__device__ __forceinline__ void slots2_t0(const double *s0, const double *s1, int G, double &o0,
                                          double &o1) {
  if (threadIdx.x < 32) {
    double v0 = 0.0, v1 = 0.0;
    for (int b = 0; b < G; b += 160) {
      double t[5], u[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const int i = b + threadIdx.x + 32 * k;
        t[k] = (i < G) ? __ldcg(s0 + i) : 0.0;
        u[k] = (i < G) ? __ldcg(s1 + i) : 0.0;
      }
      v0 += ((t[0] + t[1]) + (t[2] + t[3])) + t[4];
      v1 += ((u[0] + u[1]) + (u[2] + u[3])) + u[4];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_xor_sync(0xffffffffu, v0, o);
      v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    o0 = v0;
    o1 = v1;
  }
}

// The PCG solve (or one product in APPLY mode) of one problem by the CTAs
// cta = 0..G-1 (the whole grid, or one team of the batched solver).  The
// scalar recurrence (rho, alpha, beta, the stopping tests) runs in thread 0
// and reaches the other threads through shared memory: FP64 arithmetic is
// scarce on this SM, so it is not repeated by every warp.
template <class OP, class T>
__device__ void pcg_body(const PcgArgs &a, const int cta, const int G, unsigned char *smem,
                         double *sh, double *sbuf) {
  const int tid = threadIdx.x;
  const int64_t nkp = a.P.nkp, n = a.P.n;
  const int64_t chunk = ceil_div64(nkp, G);
  const int64_t vb = min(nkp, (int64_t)cta * chunk), ve = min(nkp, vb + chunk);
  const int vt = vec_threads(ve - vb);
  T *accg = reinterpret_cast<T *>(a.accx);
  double *pold = a.pb0, *pnew = a.pb1;
  double beta = 0.0;
  // thread 0's scalars
  double rho = 0.0, bb = 0.0, rr = 0.0, rr_mark = 0.0;
  int it = 0;
  bool ok = true, stop = false;
  const double *ysrc = a.apply ? a.rhs : a.y;
  PipeState ps;
  if constexpr (IsStaged<OP>::value) OP::template begin<T>(a, smem, ps);
  if constexpr (IsRows<OP>::value) OP::template begin<T>(a, smem);

  // ---- initialisation: z = 0, r = rhs, y = r / diag, p_old = 0
  {
    double part[2] = {0.0, 0.0};
    if (tid < vt) {
      for (int64_t i = vb + tid; i < ve; i += vt) {
        pold[i] = 0.0;
        if (a.p32_0) a.p32_0[i] = 0.f;
        if (i < n) accg[i] = (T)0;
        if (!a.apply) {
          const double ri = a.rhs[i];
          const double di = 1.0 / a.diag[i];
          if (a.dinv) a.dinv[i] = di;
          const double yi = ri * di;
          a.z[i] = 0.0;
          a.r[i] = ri;
          a.y[i] = yi;
          if (a.y32) a.y32[i] = (float)yi;
          part[0] += ri * ri;
          part[1] += ri * yi;
        }
      }
    }
    if (cta == 0 && a.g)
      for (int64_t c = tid; c < a.P.k + a.P.me; c += blockDim.x) a.g[c] = 0.0;
    vec_sum<2>(part, sh, vt);
    if (tid == 0) { a.slots[cta] = part[0]; a.slots[G + cta] = part[1]; }
  }
  ok = grid_sync(a.bar);
  if (ok && !a.apply) {
    slots2_t0(a.slots, a.slots + G, G, bb, rho);
    if (tid == 0) {
      rr = bb;
      rr_mark = bb;
      sh[0] = (rr <= a.tol2 * bb || a.maxit <= 0) ? 1.0 : 0.0;
    }
    __syncthreads();
    stop = sh[0] != 0.0;
    __syncthreads();
  }
  while (ok) {
    if (!a.apply && stop) break;
    // ---- phase A: q = K p,  p = y + beta p_old
    double pq = run_phaseA<OP, T>(a, ysrc, pold, pnew, beta, vb, ve, smem, ps, ok, cta, G);
    if (!ok) break;
    pq = block_sum_buf(pq, sbuf, sh);
    if (tid == 0) a.slots[2 * G + cta] = pq;
    ok = grid_sync(a.bar);
    if (!ok) break;
    if (a.apply) {
      if (tid < vt)
        for (int64_t i = vb + tid; i < ve; i += vt) {
          const double pi = pnew[i];
          a.z[i] = (i < n) ? (double)__ldcg(accg + i) + a.dg[i] * pi : __ldcg(a.qlam + (i - n));
        }
      break;
    }
    // the owned entries' operands do not depend on alpha: with at most one
    // owned entry per vector thread, load them before the slot sum so that the
    // two memory round trips overlap
    const bool one_each = (ve - vb) <= (int64_t)vt;
    const int64_t ci = vb + tid;
    const bool mine = one_each && tid < vt && ci < ve;
    double c_p = 0.0, c_q = 0.0, c_z = 0.0, c_r = 0.0, c_di = 0.0;
    if (mine) {
      c_p = pnew[ci];
      c_q = (ci < n) ? (double)__ldcg(accg + ci) + a.dg[ci] * c_p : __ldcg(a.qlam + (ci - n));
      c_z = a.z[ci];
      c_r = a.r[ci];
      c_di = a.dinv ? a.dinv[ci] : 1.0 / a.diag[ci];
    }
    // alpha = rho / p'Kp (thread 0)
    {
      double pqt = 0.0, unused = 0.0;
      if (tid < 32) pqt = slot_sum_w0(a.slots + 2 * G, G);
      (void)unused;
      if (tid == 0) {
        const int bad = (pqt > 0.0) ? 0 : (isnan(pqt) ? 8 : 4);
        if (bad && cta == 0) atomicCAS(a.bar.err, 0, bad);
        sh[0] = bad ? 0.0 : rho / pqt;
        sh[1] = (double)bad;
        if (a.lanczos && cta == 0 && it < a.lanczos_cap) a.lanczos[2 * it] = sh[0];
      }
      __syncthreads();
      const double alpha = sh[0];
      const bool bad = sh[1] != 0.0;
      __syncthreads();
      if (bad) break;
      // ---- phase C: vector updates on owned entries
      double part[2] = {0.0, 0.0};
      if (one_each) {
        if (mine) {
          if (ci < n) accg[ci] = (T)0;
          a.z[ci] = c_z + alpha * c_p;
          const double ri = c_r - alpha * c_q;
          a.r[ci] = ri;
          const double yi = ri * c_di;
          a.y[ci] = yi;
          if (a.y32) a.y32[ci] = (float)yi;
          part[0] = ri * ri;
          part[1] = ri * yi;
        }
      } else if (tid < vt) {
        for (int64_t i = vb + tid; i < ve; i += vt) {
          const double pi = pnew[i];
          double qi;
          if (i < n) {
            qi = (double)__ldcg(accg + i) + a.dg[i] * pi;
            accg[i] = (T)0;
          } else {
            qi = __ldcg(a.qlam + (i - n));
          }
          a.z[i] += alpha * pi;
          const double ri = a.r[i] - alpha * qi;
          a.r[i] = ri;
          const double yi = a.dinv ? ri * a.dinv[i] : ri / a.diag[i];
          a.y[i] = yi;
          if (a.y32) a.y32[i] = (float)yi;
          part[0] += ri * ri;
          part[1] += ri * yi;
        }
      }
      if (cta == 0 && a.g)
        for (int64_t c = tid; c < a.P.k + a.P.me; c += blockDim.x) a.g[c] = 0.0;
      vec_sum<2>(part, sh, vt);
      if (tid == 0) { a.slots[cta] = part[0]; a.slots[G + cta] = part[1]; }
    }
    ok = grid_sync(a.bar);
    if (!ok) break;
    // beta and the stopping tests (thread 0)
    {
      double rho_new = 0.0, rrn = 0.0;
      slots2_t0(a.slots, a.slots + G, G, rrn, rho_new);
      if (tid == 0) {
        rr = rrn;
        const double bt = rho_new / rho;
        if (a.lanczos && cta == 0 && it < a.lanczos_cap) a.lanczos[2 * it + 1] = bt;
        rho = rho_new;
        bool st = rr <= a.tol2 * bb || it + 1 >= a.maxit;
        // FP32 correction passes: hand over to the FP64 pass once they stagnate
        if (!st && a.stag_window > 0 && (it + 1) % a.stag_window == 0) {
          if (rr > 0.25 * rr_mark) st = true;
          rr_mark = rr;
        }
        sh[0] = bt;
        sh[1] = st ? 1.0 : 0.0;
      }
      __syncthreads();
      beta = sh[0];
      stop = sh[1] != 0.0;
      __syncthreads();
    }
    double *t = pold; pold = pnew; pnew = t;
    ++it;
  }
  if constexpr (IsStaged<OP>::value) OP::drain(a, smem, ps);
  if (cta == 0 && tid == 0) {
    *a.iters = it;
    a.resn[0] = rr;
    a.resn[1] = bb;
  }
}

template <class OP, class T>
__global__ void __launch_bounds__(512, 1) pcg_kernel(PcgArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[32 * 2];
  __shared__ double sbuf[512];
  pcg_body<OP, T>(a, blockIdx.x, gridDim.x, smem, sh, sbuf);
}

// the same with 256 threads (the FP64 register-streamed products: half the
// warps, each with twice the registers)
template <class OP, class T>
__global__ void __launch_bounds__(256, 1) pcg_kernel_256(PcgArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[32 * 2];
  __shared__ double sbuf[512];
  pcg_body<OP, T>(a, blockIdx.x, gridDim.x, smem, sh, sbuf);
}

// Batched dense PCG: CTA b belongs to team cta_team[b]; a team works through
// its list of problems one after another, each with pcg_body on the team's
// CTAs (team-local bounded barrier in that problem's GridBar).
struct TeamInfo { int first_cta, size, qp_begin, qp_end; };

template <class HS, class AS, class T>
__global__ void __launch_bounds__(512, 1) pcg_batch_kernel(const PcgArgs *__restrict__ args,
                                                            const int *__restrict__ cta_team,
                                                            const TeamInfo *__restrict__ teams,
                                                            const int *__restrict__ team_qps) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[32 * 2];
  __shared__ double sbuf[512];
  const int tix = cta_team[blockIdx.x];
  if (tix < 0) return;              // a CTA the device-side plan left idle
  const TeamInfo ti = teams[tix];
  const int rank = blockIdx.x - ti.first_cta;
  for (int q = ti.qp_begin; q < ti.qp_end; ++q) {
    const PcgArgs &aq = args[team_qps[q]];
    if (!aq.run) continue;          // uniform over the team: written before the launch
    pcg_body<OpDense<HS, AS>, T>(aq, rank, ti.size, smem, sh, sbuf);
    __syncthreads();
  }
}

// The captured graph's correction pass: one launch in which each problem's
// team runs it in the precision its control word chose (FP32 arguments in
// args32, FP64 in args64; run flags set on the device before the launch).
template <class HS, class AS>
__global__ void __launch_bounds__(512, 1) pcg_batch_kernel_dual(const PcgArgs *__restrict__ args32,
                                                                 const PcgArgs *__restrict__ args64,
                                                                 const int *__restrict__ cta_team,
                                                                 const TeamInfo *__restrict__ teams,
                                                                 const int *__restrict__ team_qps) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[32 * 2];
  __shared__ double sbuf[512];
  const int tix = cta_team[blockIdx.x];
  if (tix < 0) return;              // a CTA the device-side plan left idle
  const TeamInfo ti = teams[tix];
  const int rank = blockIdx.x - ti.first_cta;
  for (int q = ti.qp_begin; q < ti.qp_end; ++q) {
    const int j = team_qps[q];
    if (args32[j].run) pcg_body<OpDense<HS, AS>, float>(args32[j], rank, ti.size, smem, sh, sbuf);
    else if (args64[j].run) pcg_body<OpDense<HS, AS>, double>(args64[j], rank, ti.size, smem, sh, sbuf);
    else continue;
    __syncthreads();
  }
}

// column window [lo, hi) of each CTA's row range (CSR)
__global__ void k_windows(const int64_t *rowptr, const int32_t *col, const int64_t *row_begin,
                          int32_t *lo, int32_t *hi) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const int64_t s = rowptr[row_begin[c]], e = rowptr[row_begin[c + 1]];
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t k = s + threadIdx.x; k < e; k += blockDim.x) {
    const double v = (double)col[k];
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  mn = block_min(mn, sh);
  mx = -block_min(-mx, sh);
  if (threadIdx.x == 0) {
    if (e > s) { lo[c] = (int32_t)mn; hi[c] = (int32_t)mx + 1; }
    else { lo[c] = 0; hi[c] = 0; }
  }
}

__global__ void k_axpy_res(int64_t N, const double *rhs, const double *kz, double *res,
                           double *part) {
  __shared__ double sh[32];
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = rhs[i] - kz[i];
    res[i] = v;
    s[0] += v * v;
  }
  block_sum<1>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_sumsq(int64_t N, const double *v, double *part) {
  __shared__ double sh[32];
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    s[0] += v[i] * v[i];
  block_sum<1>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_add(int64_t N, double *z, const double *dz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] += dz[i];
}

__global__ void k_final_sum(int nb, const double *part, double *out) {
  __shared__ double sh[32];
  double s[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s[0] += part[i];
  block_sum<1>(s, sh);
  if (threadIdx.x == 0) *out = s[0];
}

using KFun = void (*)(PcgArgs);

template <class T> KFun pick_kernel(const DevProb &P) {
  if (P.hkind == KQ_H_CSR_LSQ) return pcg_kernel<OpCsrStaged, T>;
  if (P.hkind == KQ_H_LOWRANK) {
    if (P.hdtype == KQ_F64) return pcg_kernel<OpLowrank<double>, T>;
    return pcg_kernel<OpLowrank<float>, T>;
  }
  // DENSE
  const bool a64 = P.adtype == KQ_F64;
  if (P.hdtype == KQ_F64) return a64 ? pcg_kernel<OpDense<double, double>, T> : pcg_kernel<OpDense<double, float>, T>;
  if (P.hdtype == KQ_F32) return a64 ? pcg_kernel<OpDense<float, double>, T> : pcg_kernel<OpDense<float, float>, T>;
  return a64 ? pcg_kernel<OpDense<__nv_bfloat16, double>, T> : pcg_kernel<OpDense<__nv_bfloat16, float>, T>;
}


RowDesc split_w2(int32_t off, int32_t a, double w2) {
  const float hi = (float)w2;
  const float lo = (float)(w2 - (double)hi);
  return RowDesc{off, a, hi, lo};
}

template <class X> X *dalloc(kq_problem *h, size_t count) {
  void *p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(X)) != cudaSuccess) return nullptr;
  h->allocs.push_back(p);
  return reinterpret_cast<X *>(p);
}

kq_status launch(kq_problem *h, int prec, const double *rhs, double *z, double tol, int maxit,
                 int apply, int *iters_out, double *rr_out, double *bb_out) {
  PcgWork &W = h->W;
  PcgArgs a{};
  a.P = h->P;
  a.Dl = h->K.Dl; a.Du = h->K.Du; a.cl = h->K.cl; a.cu = h->K.cu;
  a.dg = h->K.dg; a.diag = h->K.diag; a.mu = h->K.mu;
  a.rhs = rhs; a.z = z;
  a.r = W.r; a.y = W.y; a.pb0 = W.pb0; a.pb1 = W.pb1; a.qlam = W.qlam;
  a.accx = prec == KQ_PREC_MIXED ? (void *)W.accx32 : (void *)W.accx64;
  a.g = (h->P.hkind == KQ_H_LOWRANK) ? W.g64 : nullptr;
  a.slots = W.slots;
  a.row_begin = W.row_begin; a.win_lo = W.win_lo; a.win_hi = W.win_hi; a.win_cap = W.win_cap;
  a.bar.count = W.bar; a.bar.gen = W.bar + 1; a.bar.err = W.err; a.bar.nblocks = W.G;
  a.bar.budget_ns = (uint64_t)(h->timeout_s * 1e9);
  a.tol2 = tol * tol; a.maxit = maxit; a.apply = apply;
  a.iters = W.iters; a.resn = W.resn;
  a.chunks = W.chunks; a.cta_chunk = W.cta_chunk; a.rdesc = W.rdesc;
  a.a_lo = W.a_lo; a.a_hi = W.a_hi;
  a.a_cap = W.a_cap; a.ch_cap = W.ch_cap; a.desc_cap = W.desc_cap; a.tab_cap = W.tab_cap;
  a.copy_piece = W.copy_piece;
  a.stages = W.stages;
  a.producer = W.producer;
  a.stag_window = (prec == KQ_PREC_MIXED && !apply) ? W.stag_window : 0;
  a.coefA = W.coefA;
  a.rslot = W.rslot;
  a.rval4 = reinterpret_cast<const float4 *>(W.rval);
  a.rcol2 = reinterpret_cast<const uint2 *>(W.rcol);
  a.rws = W.rws;
  a.pf_dist = W.pf_dist;
  KFun f = prec == KQ_PREC_MIXED ? pick_kernel<float>(h->P) : pick_kernel<double>(h->P);
  size_t smem = W.smem;
  int threads = W.threads;
  a.dinv = W.dinv;
  a.rw2lo = W.rw2lo;
  if (h->lz_on && !apply) {
    a.lanczos = W.lanczos;
    a.lanczos_cap = KQ_LANCZOS_CAP;
  }
  if (prec == KQ_PREC_MIXED && W.rows_ok) {
    f = pcg_kernel<OpCsrRows, float>;
    smem = W.smem_rows;
    a.p32_0 = W.p32_0; a.p32_1 = W.p32_1; a.y32 = W.y32;
  } else if (prec == KQ_PREC_F64 && W.rows_ok && W.rows64_ok) {
    f = pcg_kernel_256<OpCsrRows, double>;
    smem = W.smem_rows64;
    threads = W.threads_rows64;
  }
  KQ_CUDA(h, cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  KQ_CUDA(h, cudaMemsetAsync(W.err, 0, sizeof(int), h->stream));
  KQ_CUDA(h, cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned int), h->stream));
  void *args[] = {&a};
  KQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  KQ_CUDA(h, cudaLaunchCooperativeKernel((const void *)f, dim3(W.G), dim3(threads), args,
                                         smem, h->stream));
  ++h->launches;
  ++h->pcg_launches;
  KQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  // status words back to the host
  KQ_CUDA(h, cudaMemcpyAsync(W.h_pinned, W.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  KQ_CUDA(h, cudaMemcpyAsync(W.h_pinned + 1, W.iters, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  KQ_CUDA(h, cudaMemcpyAsync(W.h_pinned + 2, W.resn, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  KQ_CUDA(h, cudaEventElapsedTime(&h->last_kernel_ms, h->ev0, h->ev1));
  const int err = W.h_pinned[0];
  if (iters_out) *iters_out = W.h_pinned[1];
  double rb[2];
  memcpy(rb, W.h_pinned + 2, sizeof rb);
  if (rr_out) *rr_out = rb[0];
  if (bb_out) *bb_out = rb[1];
  if (err == 7) return kq_fail(h, KQ_ERR_TIMEOUT, "PCG grid barrier exceeded its time budget");
  if (err == 4) return kq_fail(h, KQ_ERR_NOT_CONVEX, "PCG met p'Kp <= 0 (K not positive definite)");
  if (err == 8) return kq_fail(h, KQ_ERR_NUMERIC, "PCG met NaN");
  if (err != 0) return kq_fail(h, KQ_ERR_CUDA, "PCG kernel error flag " + std::to_string(err));
  return KQ_OK;
}

double dev_norm(kq_problem *h, const double *v, int64_t N) {
  const int nb = 256;
  k_sumsq<<<nb, 256, 0, h->stream>>>(N, v, h->red);
  ++h->launches;
  k_final_sum<<<1, 256, 0, h->stream>>>(nb, h->red, h->red_out);
  ++h->launches;
  cudaMemcpyAsync(h->h_red, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  return sqrt(h->h_red[0]);
}

}  // namespace

// Persistent PCG on a dense problem whose blocks and work buffers the caller
// supplies (device pointers); launches, copies two status words back, and
// allocates nothing.
kq_status pcg_dense_raw(const DevProb &P, const double *Dl, const double *Du, const double *cl,
                        const double *cu, const double *dg, const double *diag, const double *rhs,
                        double *z, const PcgRawWork &w, int G, double tol, int maxit,
                        double timeout_s, cudaStream_t stream, int *iters, double *rr,
                        double *bb, std::string *msg) {
  PcgArgs a{};
  a.P = P;
  a.Dl = Dl; a.Du = Du; a.cl = cl; a.cu = cu; a.dg = dg; a.diag = diag; a.mu = 1.0;
  a.rhs = rhs; a.z = z;
  a.r = w.r; a.y = w.y; a.pb0 = w.pb0; a.pb1 = w.pb1; a.qlam = w.qlam;
  a.accx = w.accx; a.g = nullptr; a.slots = w.slots;
  a.row_begin = nullptr; a.win_lo = nullptr; a.win_hi = nullptr;
  a.win_cap = (int)((P.n + 7) & ~(int64_t)7);
  a.bar.count = w.bar; a.bar.gen = w.bar + 1; a.bar.err = w.err; a.bar.nblocks = (unsigned)G;
  a.bar.budget_ns = (uint64_t)(timeout_s * 1e9);
  a.tol2 = tol * tol; a.maxit = maxit; a.apply = 0;
  a.iters = w.iters; a.resn = w.resn;
  a.stages = 2; a.producer = 0; a.copy_piece = 16;
  KFun f = pcg_kernel<OpDense<double, double>, double>;
  const size_t smem = (size_t)2 * a.win_cap * sizeof(double);
  const int threads = 512;
  auto fail = [&](const char *what, cudaError_t e) {
    if (msg) *msg = std::string(what) + ": " + cudaGetErrorString(e);
    return KQ_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return fail("cudaFuncSetAttribute", e);
  void *args[] = {&a};
  if ((e = cudaLaunchCooperativeKernel((const void *)f, dim3(G), dim3(threads), args, smem, stream)) != cudaSuccess)
    return fail("cudaLaunchCooperativeKernel", e);
  int hs[2] = {0, 0};
  double hr[2] = {0.0, 0.0};
  if ((e = cudaMemcpyAsync(&hs[0], w.err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&hs[1], w.iters, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(hr, w.resn, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return fail("status read-back", e);
  if (iters) *iters = hs[1];
  if (rr) *rr = hr[0];
  if (bb) *bb = hr[1];
  if (hs[0] == 7) { if (msg) *msg = "grid barrier exceeded its time budget"; return KQ_ERR_TIMEOUT; }
  if (hs[0] == 4) { if (msg) *msg = "p'Kp <= 0 (K not positive definite)"; return KQ_ERR_NOT_CONVEX; }
  if (hs[0] == 8) { if (msg) *msg = "NaN in PCG"; return KQ_ERR_NUMERIC; }
  if (hs[0] != 0) { if (msg) *msg = "PCG error flag"; return KQ_ERR_CUDA; }
  return KQ_OK;
}

// ---------------------------------------------------------------- batched dense PCG
namespace {
template <class X> X *balloc(std::vector<void *> &allocs, size_t count) {
  void *p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(X)) != cudaSuccess) return nullptr;
  allocs.push_back(p);
  return reinterpret_cast<X *>(p);
}
}  // namespace

kq_status batch_pcg_setup(BatchPcg &B, int nqp, int sms, int max_n, std::string &err) {
  B.nqp = nqp;
  B.G = sms;   // one CTA per SM (512 threads, ~100 registers each)
  B.max_n = max_n;
  B.args = balloc<unsigned char>(B.allocs, (size_t)nqp * sizeof(PcgArgs));
  B.cta_team = balloc<int>(B.allocs, B.G);
  B.teams = balloc<unsigned char>(B.allocs, (size_t)B.G * sizeof(TeamInfo));
  B.team_qps = balloc<int>(B.allocs, nqp);
  B.d_iters = balloc<int>(B.allocs, nqp);
  B.d_err = balloc<int>(B.allocs, nqp);
  B.d_resn = balloc<double>(B.allocs, 2 * (size_t)nqp);
  if (!B.args || !B.cta_team || !B.teams || !B.team_qps || !B.d_iters || !B.d_err || !B.d_resn) {
    err = "batch PCG work space";
    return KQ_ERR_OOM;
  }
  if (cudaMallocHost((void **)&B.h_status, (size_t)nqp * (2 * sizeof(int) + 2 * sizeof(double))) != cudaSuccess) {
    err = "batch pinned status";
    return KQ_ERR_OOM;
  }
  if (cudaEventCreate(&B.ev0) != cudaSuccess || cudaEventCreate(&B.ev1) != cudaSuccess) {
    err = "batch events";
    return KQ_ERR_CUDA;
  }
  return KQ_OK;
}

void batch_pcg_free(BatchPcg &B) {
  for (void *p : B.allocs) cudaFree(p);
  B.allocs.clear();
  if (B.h_status) cudaFreeHost(B.h_status);
  B.h_status = nullptr;
  if (B.ev0) cudaEventDestroy(B.ev0);
  if (B.ev1) cudaEventDestroy(B.ev1);
  B.ev0 = B.ev1 = nullptr;
}

// Teams of CTAs for one batched launch over the listed problems: a problem
// whose share of the total cost (bytes per product times its expected
// products) is worth two or more CTAs gets a team of that size; the rest are
// packed onto single-CTA teams, largest first onto the least-loaded team.
struct TeamPlan {
  std::vector<TeamInfo> teams;
  std::vector<int> cta_team, team_qps, team_of;
  int nblocks = 0;
};

int size_bucket(int64_t n, int nb) {
  int b = 0;
  while ((int64_t(2) << b) <= n && b + 1 < nb) ++b;
  return b;
}

// cost of one K*v product of a batched problem: the autotuner's measured
// one-CTA time of its size bucket, else its bytes
double unit_cost(const kq_problem *h, const BatchTune *tune) {
  if (tune && !tune->t_prod_us.empty())
    return tune->t_prod_us[size_bucket(h->n, (int)tune->t_prod_us.size())];
  const double hb = h->P.hdtype == KQ_F64 ? 8.0 : (h->P.hdtype == KQ_F32 ? 4.0 : 2.0);
  const double ab = h->P.adtype == KQ_F64 ? 8.0 : 4.0;
  return hb * h->n * h->n + ab * h->m * h->n + 64.0 * h->nkp;
}

bool batch_f32_pays(const kq_problem *h) {
  const double hb = h->P.hdtype == KQ_F64 ? 8.0 : (h->P.hdtype == KQ_F32 ? 4.0 : 2.0);
  const double ab = h->P.adtype == KQ_F64 ? 8.0 : 4.0;
  // KQ_BATCH_F32_MIN_BYTES overrides the threshold (0: FP32 passes for every QP)
  const char *ev = getenv("KQ_BATCH_F32_MIN_BYTES");
  const double thr = ev ? atof(ev) : KQ_BATCH_F32_MIN_BYTES;
  return hb * h->n * h->n + ab * h->m * h->n >= thr;
}

// largest team of a batched problem: two rows of H, A, C per warp of the
// team, the CTAs its slot buffer holds, and the tuned cap of its size bucket
int team_cap(const kq_problem *h, const BatchTune *tune) {
  int t = (int)std::min<int64_t>(ceil_div64(h->n + h->m + h->me, 32), h->num_sms);
  if (tune && !tune->team_cap.empty())
    t = std::min(t, tune->team_cap[size_bucket(h->n, (int)tune->team_cap.size())]);
  return std::max(t, 1);
}

TeamPlan plan_teams(int G, const std::vector<kq_problem *> &hs, const std::vector<int> &idx,
                    const std::vector<double> *weight, const BatchTune *tune = nullptr) {
  const int k = (int)idx.size();
  TeamPlan tp;
  // ---- costs: cost per product times the expected number of products
  std::vector<double> cost(k);
  double total = 0.0;
  for (int j = 0; j < k; ++j) {
    cost[j] = unit_cost(hs[idx[j]], tune) * (weight ? std::max(1.0, (*weight)[j]) : 1.0);
    total += cost[j];
  }
  std::vector<int> order(k);
  for (int j = 0; j < k; ++j) order[j] = j;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<TeamInfo> teams;
  std::vector<std::vector<int>> members;
  int used = 0;
  size_t q = 0;
  for (; q < order.size(); ++q) {
    const int j = order[q];
    int t = (int)std::floor(G * cost[j] / total);
    const kq_problem *hj = hs[idx[j]];
    t = std::min(t, team_cap(hj, tune));
    if (tune && tune->force_team > 0 && k == 1) t = std::min(tune->force_team, hj->num_sms);
    // keep one CTA for the problems packed onto single CTAs, unless none is
    // left to pack; a team that does not fit is shrunk, not dropped (a
    // dropped problem would run on one CTA)
    const int room = (q + 1 < order.size()) ? G - 1 - used : G - used;
    t = std::min(t, room);
    if (t < 2) break;
    teams.push_back(TeamInfo{used, t, 0, 0});
    members.push_back({j});
    used += t;
  }
  const int nsingle = (q < order.size()) ? std::max(1, G - used) : 0;
  const int first_single = (int)teams.size();
  std::vector<double> load(nsingle, 0.0);
  for (int c = 0; c < nsingle; ++c) {
    teams.push_back(TeamInfo{used + c, 1, 0, 0});
    members.push_back({});
  }
  for (; q < order.size(); ++q) {
    const int j = order[q];
    int best = 0;
    for (int c = 1; c < nsingle; ++c) if (load[c] < load[best]) best = c;
    load[best] += cost[j];
    members[first_single + best].push_back(j);
  }
  const int nblocks = used + nsingle;
  std::vector<int> &cta_team = tp.cta_team, &team_qps = tp.team_qps;
  cta_team.assign(nblocks, 0);
  for (size_t t = 0; t < teams.size(); ++t) {
    teams[t].qp_begin = (int)team_qps.size();
    for (int j : members[t]) team_qps.push_back(j);
    teams[t].qp_end = (int)team_qps.size();
    for (int c = 0; c < teams[t].size; ++c) cta_team[teams[t].first_cta + c] = (int)t;
  }
  tp.team_of.assign(k, 0);
  for (size_t t = 0; t < teams.size(); ++t)
    for (int j : members[t]) tp.team_of[j] = (int)t;
  tp.teams = teams;
  tp.nblocks = nblocks;
  return tp;
}

// One launch: PCG solves (apply = 0) or single K*v products (apply = 1) of the
// listed problems.  Teams: problems whose share of the total cost is worth
// two or more CTAs get their own team of that size; the rest are packed onto
// single-CTA teams, largest first onto the least-loaded team.
kq_status batch_pcg_launch(BatchPcg &B, const std::vector<kq_problem *> &hs,
                           const std::vector<int> &idx, const std::vector<const double *> &rhs,
                           const std::vector<double *> &out, const std::vector<double> &tol,
                           const std::vector<int> &maxit, int apply, int prec, cudaStream_t s,
                           std::vector<int> &iters, std::vector<int> &errs,
                           std::vector<double> &rr, std::vector<double> &bb, float *ms,
                           std::string &err, const std::vector<double> *weight) {
  const int k = (int)idx.size();
  iters.assign(k, 0); errs.assign(k, 0); rr.assign(k, 0.0); bb.assign(k, 0.0);
  if (k == 0) { if (ms) *ms = 0.f; return KQ_OK; }
  const TeamPlan tp = plan_teams(B.G, hs, idx, weight, &B.tune);
  const std::vector<TeamInfo> &teams = tp.teams;
  const int nblocks = tp.nblocks;
  const std::vector<int> &cta_team = tp.cta_team, &team_qps = tp.team_qps;
  // ---- per-problem arguments
  std::vector<PcgArgs> args(k);
  const std::vector<int> &team_of = tp.team_of;
  size_t smem = 0;
  for (int j = 0; j < k; ++j) {
    kq_problem *h = hs[idx[j]];
    PcgWork &W = h->W;
    PcgArgs &a = args[j];
    a = PcgArgs{};
    a.P = h->P;
    a.Dl = h->K.Dl; a.Du = h->K.Du; a.cl = h->K.cl; a.cu = h->K.cu;
    a.dg = h->K.dg; a.diag = h->K.diag; a.mu = h->K.mu;
    a.rhs = rhs[j]; a.z = out[j];
    a.r = W.r; a.y = W.y; a.pb0 = W.pb0; a.pb1 = W.pb1; a.qlam = W.qlam;
    a.accx = prec == KQ_PREC_MIXED ? (void *)W.accx32 : (void *)W.accx64;
    a.g = nullptr; a.slots = W.slots;
    a.win_cap = (int)((h->n + 7) & ~(int64_t)7);
    a.bar.count = W.bar; a.bar.gen = W.bar + 1; a.bar.err = B.d_err + j;
    a.bar.nblocks = (unsigned)teams[team_of[j]].size;
    a.bar.budget_ns = (uint64_t)(h->timeout_s * 1e9);
    a.tol2 = tol[j] * tol[j]; a.maxit = maxit[j]; a.apply = apply;
    a.iters = B.d_iters + j; a.resn = B.d_resn + 2 * j;
    a.stages = 2; a.producer = 0; a.copy_piece = 16;
    a.stag_window = (prec == KQ_PREC_MIXED && !apply) ? W.stag_window : 0;
    a.coefA = W.coefA;
    a.dinv = W.dinv;
    a.run = 1;
    a.colpass_min_n = B.tune.colpass_min_n;
    smem = std::max(smem, (size_t)2 * a.win_cap * (prec == KQ_PREC_MIXED ? sizeof(float) : sizeof(double)));
    if (cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) { err = "memset"; return KQ_ERR_CUDA; }
  }
  const kq_problem *h0 = hs[idx[0]];
  for (int j = 1; j < k; ++j) {
    const kq_problem *h = hs[idx[j]];
    if (h->P.hdtype != h0->P.hdtype || h->P.adtype != h0->P.adtype || h->P.hkind != KQ_H_DENSE) {
      err = "batched problems must share the dense H and A storage types";
      return KQ_ERR_ARG;
    }
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(B.d_err, 0, k * sizeof(int), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(B.args, args.data(), k * sizeof(PcgArgs), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(B.cta_team, cta_team.data(), nblocks * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(B.teams, teams.data(), teams.size() * sizeof(TeamInfo), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(B.team_qps, team_qps.data(), team_qps.size() * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    err = std::string("batch upload: ") + cudaGetErrorString(e);
    return KQ_ERR_CUDA;
  }
  const void *f;
  const bool mixed = prec == KQ_PREC_MIXED;
  if (h0->P.hdtype == KQ_BF16 && h0->P.adtype == KQ_F32)
    f = mixed ? (const void *)pcg_batch_kernel<__nv_bfloat16, float, float>
              : (const void *)pcg_batch_kernel<__nv_bfloat16, float, double>;
  else if (h0->P.hdtype == KQ_F64 && h0->P.adtype == KQ_F64)
    f = mixed ? (const void *)pcg_batch_kernel<double, double, float>
              : (const void *)pcg_batch_kernel<double, double, double>;
  else {
    err = "batched PCG supports bf16 H with f32 A, or f64 H with f64 A";
    return KQ_ERR_ARG;
  }
  if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
    err = std::string("batch attribute: ") + cudaGetErrorString(e);
    return KQ_ERR_CUDA;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 512, smem);
  if (per_sm * B.G < nblocks) { err = "batched PCG grid does not fit"; return KQ_ERR_ARG; }
  const PcgArgs *pa = reinterpret_cast<const PcgArgs *>(B.args);
  const TeamInfo *pt = reinterpret_cast<const TeamInfo *>(B.teams);
  void *kargs[] = {(void *)&pa, (void *)&B.cta_team, (void *)&pt, (void *)&B.team_qps};
  cudaEventRecord(B.ev0, s);
  if ((e = cudaLaunchCooperativeKernel(f, dim3(nblocks), dim3(512), kargs, smem, s)) != cudaSuccess) {
    err = std::string("batch launch: ") + cudaGetErrorString(e);
    return KQ_ERR_CUDA;
  }
  cudaEventRecord(B.ev1, s);
  B.launches++;
  int *hi = reinterpret_cast<int *>(B.h_status);
  int *he = hi + B.nqp;
  double *hr = reinterpret_cast<double *>(he + B.nqp);
  if ((e = cudaMemcpyAsync(hi, B.d_iters, k * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(he, B.d_err, k * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(hr, B.d_resn, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    err = std::string("batch status: ") + cudaGetErrorString(e);
    return KQ_ERR_CUDA;
  }
  float t = 0.f;
  cudaEventElapsedTime(&t, B.ev0, B.ev1);
  if (ms) *ms = t;
  for (int j = 0; j < k; ++j) {
    iters[j] = hi[j]; errs[j] = he[j]; rr[j] = hr[2 * j]; bb[j] = hr[2 * j + 1];
  }
  return KQ_OK;
}

double pcg_last_kernel_ms(const kq_problem *h) { return h->last_kernel_ms; }

// Self-test of the bounded device waits: every CTA enters the production grid
// barrier once with an arrival target one above the CTAs launched, so the
// barrier cannot complete; each wait gives up after its budget and records
// KQ_ERR_TIMEOUT.
namespace {
__global__ void k_barrier_selftest(GridBar g, int *done) {
  const bool ok = grid_sync(g);
  if (threadIdx.x == 0 && !ok) atomicAdd(done, 1);
}
}  // namespace

extern "C" kq_status kq_barrier_selftest(int ctas, double budget_s, int *gave_up,
                                         double *elapsed_ms) {
  if (ctas < 1 || ctas > 1024 || !(budget_s > 0.0) || budget_s > 5.0)
    return kq_fail(nullptr, KQ_ERR_ARG, "kq_barrier_selftest: 1 <= ctas <= 1024, 0 < budget <= 5 s");
  unsigned int *w = nullptr;
  if (cudaMalloc(&w, 4 * sizeof(unsigned int)) != cudaSuccess)
    return kq_fail(nullptr, KQ_ERR_OOM, "kq_barrier_selftest: work words");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  kq_status st = KQ_OK;
  int h[2] = {0, 0};
  float ms = 0.f;
  GridBar g;
  g.count = w;
  g.gen = w + 1;
  g.err = reinterpret_cast<int *>(w + 2);
  g.nblocks = (unsigned)ctas + 1u;   // never reached: nothing else arrives
  g.budget_ns = (uint64_t)(budget_s * 1e9);
  if (cudaMemset(w, 0, 4 * sizeof(unsigned int)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = kq_fail(nullptr, KQ_ERR_CUDA, "kq_barrier_selftest: set-up");
  } else {
    cudaEventRecord(e0);
    k_barrier_selftest<<<ctas, 128>>>(g, reinterpret_cast<int *>(w + 3));
    cudaEventRecord(e1);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h, w + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = kq_fail(nullptr, KQ_ERR_CUDA, "kq_barrier_selftest: launch");
    } else {
      cudaEventElapsedTime(&ms, e0, e1);
      if (gave_up) *gave_up = h[1];
      if (elapsed_ms) *elapsed_ms = ms;
      st = h[0] == 7 ? KQ_ERR_TIMEOUT : (h[0] == 0 ? KQ_OK : KQ_ERR_CUDA);
      if (st == KQ_ERR_TIMEOUT) kq_fail(nullptr, st, "grid barrier exceeded its time budget");
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(w);
  return st;
}

// Fill of the register-streamed layout, one warp per row of P.  The row's
// nonzeros are ranked by (multiplicity of their bank in the row, descending;
// bank; position) and rank i goes to lane i/4, component i%4, so entries of
// one bank are dealt to different load components.  Padding slots get value
// 0 and a window column outside the row, preferably on a bank that their
// component does not use yet.  err[0] = 1 if a row has no room for padding.
__global__ void k_rows_fill(const int64_t *rowptr, const int32_t *col, const float *val,
                            const RowSlot *slots, const int64_t *row_begin,
                            const int32_t *win_lo, const int32_t *win_hi, int G, int64_t nP,
                            float *rv, uint16_t *rc, int *err) {
  __shared__ int s_key[8][128];
  __shared__ int s_rel[8][128];
  __shared__ int s_cnt[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < nP; r += nwarps) {
    int lo_c = 0, hi_c = G;            // CTA of row r: row_begin[c] <= r < row_begin[c+1]
    while (hi_c - lo_c > 1) {
      const int mid = (lo_c + hi_c) >> 1;
      if (row_begin[mid] <= r) lo_c = mid; else hi_c = mid;
    }
    const int lo = win_lo[lo_c], wl = win_hi[lo_c] - lo;
    const int64_t s0 = rowptr[r];
    const int len = (int)(rowptr[r + 1] - s0);
    const RowSlot sl = slots[r];
    const int64_t base = 4 * (int64_t)sl.off4;
    s_cnt[wib][lane] = 0;
    __syncwarp();
    for (int e = lane; e < len; e += 32) {
      const int rel = col[s0 + e] - lo;
      s_rel[wib][e] = rel;
      atomicAdd(&s_cnt[wib][rel & 31], 1);
    }
    __syncwarp();
    for (int e = lane; e < len; e += 32) {
      const int b = s_rel[wib][e] & 31;
      s_key[wib][e] = ((32 - s_cnt[wib][b]) << 12) | (b << 7) | e;
    }
    __syncwarp();
    uint32_t used[4] = {0u, 0u, 0u, 0u};
    for (int e = lane; e < len; e += 32) {
      const int key = s_key[wib][e];
      int rank = 0;
      for (int j = 0; j < len; ++j) rank += s_key[wib][j] < key;
      const int q = rank & 3, ln = rank >> 2;
      rv[base + 4 * ln + q] = val[s0 + e];
      rc[base + 4 * ln + q] = (uint16_t)s_rel[wib][e];
      used[q] |= 1u << (s_rel[wib][e] & 31);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) used[q] = __reduce_or_sync(0xffffffffu, used[q]);
    int nrow = len;                     // s_rel[0..nrow) = columns taken in this row
    for (int i = len; i < 4 * sl.len4; ++i) {
      const int q = i & 3, ln = i >> 2;
      int pick = -1;
      for (int pass = 0; pass < 2 && pick < 0; ++pass) {
        for (int c0 = 0; c0 < wl && pick < 0; c0 += 32) {
          const int c = c0 + lane;
          bool okc = c < wl && (pass == 1 || !((used[q] >> (c & 31)) & 1u));
          if (okc)
            for (int j = 0; j < nrow; ++j)
              if (s_rel[wib][j] == c) { okc = false; break; }
          const unsigned bal = __ballot_sync(0xffffffffu, okc);
          if (bal) pick = c0 + __ffs(bal) - 1;
        }
      }
      if (pick < 0) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      if (lane == 0) {
        rv[base + 4 * ln + q] = 0.f;
        rc[base + 4 * ln + q] = (uint16_t)pick;
        s_rel[wib][nrow] = pick;
      }
      used[q] |= 1u << (pick & 31);
      ++nrow;
      __syncwarp();
    }
    __syncwarp();
  }
}

// Register-streamed CSR layout (FP32 products).  Eligible when every row has
// at most 128 nonzeros, every CTA's window leaves room for the padding
// columns, and the per-warp accumulators fit in shared memory.  Returns
// false (and leaves the staged operator in charge) otherwise.
bool build_rows_layout(kq_problem *h, int G, int threads, const std::vector<int64_t> &rb,
                       const std::vector<int64_t> &rp, const std::vector<int32_t> &lo,
                       const std::vector<int32_t> &hi, const std::vector<int32_t> &p2a,
                       const std::vector<double> &w2) {
  PcgWork &W = h->W;
  const DevProb &P = h->P;
  if (getenv("KQ_STAGED")) return false;
  const int64_t nP = P.nP;
  int wmax = 1;
  for (int c = 0; c < G; ++c) wmax = std::max(wmax, hi[c] - lo[c]);
  if (wmax > 65536) return false;     // columns are stored as 16-bit window offsets
  const int rws = (wmax + 31) & ~31;
  const int nw = threads / 32;
  const size_t smem = rows_layout(rws, nw, W.a_cap, 4).total;
  if (smem > 220 * 1024) return false;
  // FP64 products: half the warps (their private accumulators are twice as wide)
  const size_t smem64 = rows_layout(rws, nw / 2, W.a_cap, 8).total;
  std::vector<RowSlot> slots(std::max<int64_t>(nP, 1));
  int64_t tot4 = 0;
  for (int c = 0; c < G; ++c) {
    const int wl = hi[c] - lo[c];
    for (int64_t r = rb[c]; r < rb[c + 1]; ++r) {
      const int64_t len = rp[r + 1] - rp[r], len4 = (len + 3) / 4;
      if (len > 128 || 4 * len4 > wl) return false;
      slots[r] = RowSlot{(int32_t)tot4, (int32_t)len4, p2a[r], (float)w2[r]};
      tot4 += len4;
      if (tot4 > INT32_MAX / 2) return false;
    }
  }
  W.rslot = dalloc<RowSlot>(h, slots.size());
  W.rval = dalloc<float>(h, 4 * (tot4 + 1));
  W.rcol = dalloc<uint16_t>(h, 4 * (tot4 + 1));
  int *d_err = dalloc<int>(h, 1);
  if (!W.rslot || !W.rval || !W.rcol || !d_err) return false;
  if (cudaMemcpy(W.rslot, slots.data(), slots.size() * sizeof(RowSlot), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemsetAsync(d_err, 0, sizeof(int), h->stream) != cudaSuccess)
    return false;
  if (nP > 0) {
    const int blocks = (int)std::min<int64_t>(ceil_div64(nP, 8), 4096);
    k_rows_fill<<<blocks, 256, 0, h->stream>>>(P.rowptr, P.col, P.val, W.rslot, W.row_begin,
                                                W.win_lo, W.win_hi, G, nP, W.rval, W.rcol, d_err);
    ++h->launches;
  }
  int e = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess || e != 0)
    return false;
  // low parts of the FP32-split row weights (FP64 products)
  {
    std::vector<float> lo2(std::max<int64_t>(nP, 1), 0.f);
    for (int64_t r = 0; r < nP; ++r) lo2[r] = (float)(w2[r] - (double)(float)w2[r]);
    W.rw2lo = dalloc<float>(h, lo2.size());
    if (!W.rw2lo ||
        cudaMemcpy(W.rw2lo, lo2.data(), lo2.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
  }
  W.rws = rws;
  W.smem_rows = smem;
  W.rows64_ok = smem64 <= 220 * 1024;
  W.smem_rows64 = smem64;
  W.threads_rows64 = threads / 2;
  {
    const char *pf = getenv("KQ_PF");
    W.pf_dist = pf ? std::max(0, atoi(pf)) : 0;
  }
  return true;
}

kq_status pcg_setup(kq_problem *h, int grid_ctas) {
  PcgWork &W = h->W;
  const DevProb &P = h->P;
  const int64_t n = P.n, nkp = P.nkp;
  int threads = 512;
  size_t smem = 0;
  int win_cap = 0;
  if (P.hkind == KQ_H_DENSE) {
    threads = 512;
    win_cap = (int)((n + 7) & ~(int64_t)7);
    smem = (size_t)2 * win_cap * sizeof(double);
    if (smem > 200 * 1024)
      return kq_fail(h, KQ_ERR_ARG, "dense H: n too large for the single-problem kernel");
  }
  int sms = h->num_sms;
  // provisional grid for the partition
  int G = grid_ctas > 0 ? grid_ctas : sms;
  if (P.hkind == KQ_H_DENSE) {
    // small dense problems are latency-bound: fewer CTAs, cheaper barriers
    // (two rows per warp; a single CTA was measured slower on n = 200: the
    // row dots are then bound by one SM's FP64 and shuffle throughput)
    const int64_t rows = n + P.m + P.me;
    const int64_t want = ceil_div64(rows, (int64_t)(threads / 32) * 2);
    G = grid_ctas > 0 ? grid_ctas : (int)std::max<int64_t>(1, std::min<int64_t>(sms, want));
  }
  W.row_begin = dalloc<int64_t>(h, G + 1);
  W.win_lo = dalloc<int32_t>(h, G);
  W.win_hi = dalloc<int32_t>(h, G);
  if (!W.row_begin || !W.win_lo || !W.win_hi) return kq_fail(h, KQ_ERR_OOM, "pcg partition");
  std::vector<int64_t> rb(G + 1, 0);
  std::vector<int64_t> rp;
  if (P.hkind == KQ_H_CSR_LSQ) {
    rp.resize(P.nP + 1);
    KQ_CUDA(h, cudaMemcpy(rp.data(), P.rowptr, (P.nP + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    const int64_t nnz = rp[P.nP];
    for (int c = 0; c <= G; ++c) {
      const int64_t target = (nnz * c) / G;
      rb[c] = std::lower_bound(rp.begin(), rp.end(), target) - rp.begin();
      if (rb[c] > P.nP) rb[c] = P.nP;
    }
    rb[0] = 0;
    rb[G] = P.nP;
    for (int c = 1; c <= G; ++c) rb[c] = std::max(rb[c], rb[c - 1]);
  } else {
    const int64_t rows = (P.hkind == KQ_H_LOWRANK) ? n : 0;
    for (int c = 0; c <= G; ++c) rb[c] = rows * c / G;
  }
  KQ_CUDA(h, cudaMemcpy(W.row_begin, rb.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  if (P.hkind == KQ_H_CSR_LSQ) {
    k_windows<<<G, 256, 0, h->stream>>>(P.rowptr, P.col, W.row_begin, W.win_lo, W.win_hi);
    ++h->launches;
    KQ_CUDA(h, cudaGetLastError());
    std::vector<int32_t> lo(G), hi(G);
    KQ_CUDA(h, cudaMemcpyAsync(lo.data(), W.win_lo, G * 4, cudaMemcpyDeviceToHost, h->stream));
    KQ_CUDA(h, cudaMemcpyAsync(hi.data(), W.win_hi, G * 4, cudaMemcpyDeviceToHost, h->stream));
    KQ_CUDA(h, cudaStreamSynchronize(h->stream));
    // window starts on a multiple of 4 columns (16-byte aligned flushes)
    for (int c = 0; c < G; ++c) lo[c] &= ~3;
    KQ_CUDA(h, cudaMemcpy(W.win_lo, lo.data(), G * 4, cudaMemcpyHostToDevice));
    int wmax = 0;
    for (int c = 0; c < G; ++c) wmax = std::max(wmax, hi[c] - lo[c]);
    // ---- chunk tables for the staged kernel
    // ring geometry (defaults; KQ_CHUNK / KQ_STAGES / KQ_COPY_PIECE override for tuning)
    auto env_int = [](const char *k, int d) { const char *v = getenv(k); return v ? atoi(v) : d; };
    const int ch_cap = std::max(256, std::min(16384, env_int("KQ_CHUNK", 4096))) & ~3;
    W.stages = std::max(2, std::min(KQ_MAX_STAGES, env_int("KQ_STAGES", 4)));
    W.copy_piece = std::max(16, env_int("KQ_COPY_PIECE", ch_cap * 4)) & ~15;
    {
      const char *pr = getenv("KQ_PRODUCER");
      W.producer = (pr && std::string(pr) == "bulk") ? 1 : 0;
    }
    const int desc_cap = std::max(8, ch_cap / 32);  // descriptors per stage
    // two rows per warp per chunk keeps the warps of a CTA evenly loaded
    const int rows_per_chunk = std::min(desc_cap - 2, 2 * (threads / 32));
    std::vector<int32_t> p2a(P.nP);
    std::vector<double> w2(P.nP);
    KQ_CUDA(h, cudaMemcpy(p2a.data(), P.prow2a, P.nP * sizeof(int32_t), cudaMemcpyDeviceToHost));
    KQ_CUDA(h, cudaMemcpy(w2.data(), P.w2, P.nP * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<ChunkInfo> chunks;
    std::vector<RowDesc> desc;
    std::vector<int32_t> cta_chunk(G + 1, 0), alo(G, 0), ahi(G, 0);
    int max_nc = 0, a_max = 0;
    for (int c = 0; c < G; ++c) {
      cta_chunk[c] = (int32_t)chunks.size();
      int amin = INT32_MAX, amax = -1;
      int64_t r = rb[c];
      while (r < rb[c + 1]) {
        ChunkInfo ci{};
        ci.desc0 = (int32_t)desc.size();
        const int64_t s0 = rp[r];
        const int64_t s_al = s0 & ~(int64_t)3;   // 16-byte aligned start
        if (rp[r + 1] - s_al + 4 > ch_cap) {
          // over-long row: processed from global memory by the whole CTA
          desc.push_back(RowDesc{1, (int32_t)r, 0.f, 0.f});
          desc.push_back(split_w2(0, p2a[r], w2[r]));
          desc.push_back(RowDesc{0, 0, 0.f, 0.f});
          ci.src = 0;
          ci.nelem = 0;
          if (p2a[r] >= 0) { amin = std::min(amin, p2a[r]); amax = std::max(amax, p2a[r]); }
          ++r;
        } else {
          desc.push_back(RowDesc{0, -1, 0.f, 0.f});
          int nr = 0;
          while (r < rb[c + 1] && nr < rows_per_chunk && rp[r + 1] - s_al + 4 <= ch_cap) {
            desc.push_back(split_w2((int32_t)(rp[r] - s_al), p2a[r], w2[r]));
            if (p2a[r] >= 0) { amin = std::min(amin, p2a[r]); amax = std::max(amax, p2a[r]); }
            ++nr;
            ++r;
          }
          const int64_t e = rp[r];
          desc.push_back(RowDesc{(int32_t)(e - s_al), 0, 0.f, 0.f});
          desc[ci.desc0].off = nr;
          // header.w2hi = 1: every row of the chunk has at most 128 nonzeros
          bool short_rows = true;
          for (int64_t q = r - nr; q < r; ++q) short_rows = short_rows && (rp[q + 1] - rp[q] <= 128);
          desc[ci.desc0].w2hi = short_rows ? 1.f : 0.f;
          ci.src = s_al;
          ci.nelem = (int32_t)(((e - s_al) + 3) & ~(int64_t)3);
        }
        ci.ndesc = (int32_t)desc.size() - ci.desc0;
        // keep every chunk's descriptor block 16-byte aligned (RowDesc is 16 B)
        chunks.push_back(ci);
      }
      max_nc = std::max(max_nc, (int)chunks.size() - cta_chunk[c]);
      alo[c] = amax >= 0 ? amin : 0;
      ahi[c] = amax >= 0 ? amax + 1 : 0;
      a_max = std::max(a_max, ahi[c] - alo[c]);
    }
    cta_chunk[G] = (int32_t)chunks.size();
    // stages sized to the largest chunk actually built, not the cap
    int used_elems = 4, used_desc = 3;
    for (const ChunkInfo &ci : chunks) {
      used_elems = std::max(used_elems, (int)ci.nelem);
      used_desc = std::max(used_desc, (int)ci.ndesc);
    }
    W.ch_cap = (used_elems + 31) & ~31;
    W.desc_cap = (used_desc + 7) & ~7;
    W.tab_cap = std::min(max_nc, 512);
    W.a_cap = std::min(a_max, 1024);
    // shared memory: column window + A rows + chunk table + ring.  Keep the
    // whole window if possible and give the rest to ring stages (up to 8, or
    // KQ_STAGES if set); shrink the window only if two stages do not fit.
    const size_t limit = 220 * 1024;
    win_cap = wmax;
    if (!getenv("KQ_STAGES")) {
      W.stages = 2;
      while (W.stages < KQ_MAX_STAGES &&
             csr_layout(win_cap, W.a_cap, W.ch_cap, W.desc_cap, W.tab_cap, W.stages + 1).total <= limit)
        ++W.stages;
    }
    while (csr_layout(win_cap, W.a_cap, W.ch_cap, W.desc_cap, W.tab_cap, W.stages).total > limit &&
           win_cap > 0)
      win_cap = win_cap > 1024 ? win_cap - 1024 : 0;
    smem = csr_layout(win_cap, W.a_cap, W.ch_cap, W.desc_cap, W.tab_cap, W.stages).total;
    if (smem > limit) return kq_fail(h, KQ_ERR_ARG, "CSR staging ring does not fit in shared memory");
    W.chunks = dalloc<ChunkInfo>(h, chunks.size());
    W.rdesc = dalloc<RowDesc>(h, desc.size());
    W.cta_chunk = dalloc<int32_t>(h, G + 1);
    W.a_lo = dalloc<int32_t>(h, G);
    W.a_hi = dalloc<int32_t>(h, G);
    if (!W.chunks || !W.rdesc || !W.cta_chunk || !W.a_lo || !W.a_hi)
      return kq_fail(h, KQ_ERR_OOM, "chunk tables");
    KQ_CUDA(h, cudaMemcpy(W.chunks, chunks.data(), chunks.size() * sizeof(ChunkInfo), cudaMemcpyHostToDevice));
    KQ_CUDA(h, cudaMemcpy(W.rdesc, desc.data(), desc.size() * sizeof(RowDesc), cudaMemcpyHostToDevice));
    KQ_CUDA(h, cudaMemcpy(W.cta_chunk, cta_chunk.data(), (G + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    KQ_CUDA(h, cudaMemcpy(W.a_lo, alo.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice));
    KQ_CUDA(h, cudaMemcpy(W.a_hi, ahi.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice));
    W.rows_ok = build_rows_layout(h, G, threads, rb, rp, lo, hi, p2a, w2);
    cudaGetLastError();
  } else if (P.hkind == KQ_H_LOWRANK) {
    int64_t rmax = 0;
    for (int c = 0; c < G; ++c) rmax = std::max(rmax, rb[c + 1] - rb[c]);
    win_cap = (int)rmax;
    smem = (size_t)rmax * sizeof(double) + (size_t)(P.k + P.me + 1) * sizeof(double) +
           (size_t)(P.me + 1) * sizeof(double) + 64;
    if (smem > 200 * 1024) return kq_fail(h, KQ_ERR_ARG, "lowrank: too many rows per CTA");
  }
  W.G = G;
  W.threads = threads;
  {
    // FP32 passes end when |r| has not halved over this many iterations
    // (KQ_STAG_WINDOW overrides, for tuning)
    const char *sw = getenv("KQ_STAG_WINDOW");
    W.stag_window = sw ? std::max(0, atoi(sw)) : 400;
  }
  W.win_cap = win_cap;
  W.smem = smem;
  // verify co-residency for the cooperative launch
  {
    int per_sm = 0;
    const void *f = (const void *)pick_kernel<double>(P);
    KQ_CUDA(h, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    KQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem));
    if (per_sm * sms < G)
      return kq_fail(h, KQ_ERR_ARG, "persistent PCG grid does not fit on the device");
    const void *f32 = (const void *)pick_kernel<float>(P);
    KQ_CUDA(h, cudaFuncSetAttribute(f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    KQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32, threads, smem));
    if (per_sm * sms < G)
      return kq_fail(h, KQ_ERR_ARG, "persistent PCG grid (mixed) does not fit on the device");
    if (W.rows_ok) {
      const void *fr = (const void *)pcg_kernel<OpCsrRows, float>;
      KQ_CUDA(h, cudaFuncSetAttribute(fr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W.smem_rows));
      KQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fr, threads, W.smem_rows));
      if (per_sm * sms < G) W.rows_ok = false;
    }
    if (W.rows_ok && W.rows64_ok) {
      const void *fr = (const void *)pcg_kernel_256<OpCsrRows, double>;
      KQ_CUDA(h, cudaFuncSetAttribute(fr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W.smem_rows64));
      KQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fr, W.threads_rows64, W.smem_rows64));
      if (per_sm * sms < G) W.rows64_ok = false;
    }
  }
  W.r = dalloc<double>(h, nkp);
  W.y = dalloc<double>(h, nkp);
  W.pb0 = dalloc<double>(h, nkp);
  W.pb1 = dalloc<double>(h, nkp);
  W.qlam = dalloc<double>(h, nkp - n + 1);
  W.accx64 = dalloc<double>(h, n);
  W.accx32 = dalloc<float>(h, n);
  W.g64 = dalloc<double>(h, P.k + P.me + 1);
  W.coefA = dalloc<double>(h, P.m + 1);
  W.dinv = dalloc<double>(h, nkp);
  W.lanczos = dalloc<double>(h, 2 * (size_t)KQ_LANCZOS_CAP);
  if (W.rows_ok) {
    W.p32_0 = dalloc<float>(h, nkp);
    W.p32_1 = dalloc<float>(h, nkp);
    W.y32 = dalloc<float>(h, nkp);
    if (!W.p32_0 || !W.p32_1 || !W.y32) return kq_fail(h, KQ_ERR_OOM, "pcg FP32 copies");
  }
  // per-CTA partial sums: sized for the widest team the batched solver may
  // give this problem (up to every SM), not only for this problem's own grid
  W.slots = dalloc<double>(h, 4 * (size_t)std::max(G, sms));
  W.bar = dalloc<unsigned int>(h, 2);
  W.err = dalloc<int>(h, 1);
  W.iters = dalloc<int>(h, 1);
  W.resn = dalloc<double>(h, 2);
  if (!W.r || !W.y || !W.pb0 || !W.pb1 || !W.qlam || !W.accx64 || !W.accx32 || !W.g64 ||
      !W.slots || !W.bar || !W.err || !W.iters || !W.resn || !W.coefA || !W.dinv)
    return kq_fail(h, KQ_ERR_OOM, "pcg work space");
  KQ_CUDA(h, cudaMemset(W.accx64, 0, n * sizeof(double)));
  KQ_CUDA(h, cudaMemset(W.accx32, 0, n * sizeof(float)));
  KQ_CUDA(h, cudaMallocHost((void **)&W.h_pinned, 64));
  return KQ_OK;
}

kq_status pcg_apply(kq_problem *h, const double *v, double *out, int prec, float *ms) {
  kq_status st = launch(h, prec, v, out, 0.0, 0, 1, nullptr, nullptr, nullptr);
  if (ms) *ms = h->last_kernel_ms;
  return st;
}

// Extreme eigenvalues of the Lanczos tridiagonal matrix of a PCG pass (the
// PCG-Lanczos relation: T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
// T_{j,j+1} = sqrt(beta_j)/alpha_j), by Sturm-sequence bisection.  Results in
// h->lz_min, h->lz_max, h->lz_steps (0 when the pass ran no iteration).
namespace {
int sturm_count(const std::vector<double> &d, const std::vector<double> &e2, double x) {
  int c = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    q = d[i] - x - (i > 0 ? e2[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++c;
  }
  return c;
}
}  // namespace

void lanczos_extremes(kq_problem *h, int iters) {
  h->lz_steps = 0;
  h->lz_min = h->lz_max = 0.0;
  const int k = std::min(iters, (int)KQ_LANCZOS_CAP);
  if (k <= 0) return;
  std::vector<double> ab(2 * (size_t)k);
  if (cudaMemcpy(ab.data(), h->W.lanczos, ab.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return;
  std::vector<double> d(k), e2(std::max(k - 1, 1), 0.0);
  for (int j = 0; j < k; ++j) {
    const double aj = ab[2 * j], bprev = j > 0 ? ab[2 * (j - 1) + 1] : 0.0;
    if (!(aj > 0.0)) return;
    d[j] = 1.0 / aj + (j > 0 ? bprev / ab[2 * (j - 1)] : 0.0);
    if (j + 1 < k) e2[j] = ab[2 * j + 1] / (aj * aj);   // (sqrt(beta_j) / alpha_j)^2
  }
  // Gershgorin interval
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? sqrt(e2[j - 1]) : 0.0) + (j + 1 < k ? sqrt(e2[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  auto kth = [&](int target) {   // smallest x with count(x) >= target
    double a = lo, b = hi;
    for (int t = 0; t < 200 && b - a > 1e-15 * std::max(fabs(a), fabs(b)); ++t) {
      const double m = 0.5 * (a + b);
      if (sturm_count(d, e2, m) >= target) b = m; else a = m;
    }
    return 0.5 * (a + b);
  };
  h->lz_min = kth(1);
  h->lz_max = kth(k);
  h->lz_steps = k;
}

// Jacobi PCG with optional FP32-matvec correction solves and FP64 residual
// refinement:  z = 0;  repeat { solve K dz = res (FP32 products for the first
// refine_steps passes, FP64 afterwards);  z += dz;  res = rhs - K z in FP64 }
// until |res| <= tol |rhs| or the iteration budget is spent.
kq_status pcg_solve(kq_problem *h, const double *rhs, double *z, const kq_pcg_opts &o,
                    kq_pcg_stats *st) {
  const int64_t N = h->P.nkp;
  kq_pcg_stats s{};
  const bool warm = h->warm_next;   // one solve only
  h->warm_next = false;
  const double bn = dev_norm(h, rhs, N);
  if (!(bn > 0.0)) {
    KQ_CUDA(h, cudaMemsetAsync(z, 0, N * sizeof(double), h->stream));
    s.status = (bn == 0.0) ? KQ_OK : KQ_ERR_NUMERIC;
    if (st) *st = s;
    return s.status == KQ_OK ? KQ_OK : kq_fail(h, KQ_ERR_NUMERIC, "rhs has NaN/Inf");
  }
  double *res = h->tmp, *dz = h->zref;
  double resn = bn;
  bool cold = !warm;
  if (warm) {
    // warm start from the direction already in z: res = rhs - K z in FP64
    float ms = 0.f;
    const kq_status rc0 = pcg_apply(h, z, dz, KQ_PREC_F64, &ms);
    if (rc0 != KQ_OK) return rc0;
    s.kernel_ms += ms;
    s.kernel_ms_f64 += ms;
    s.products_f64 += 1;
    s.products += 1;
    s.launches_f64 += 1;
    const int nb = 256;
    k_axpy_res<<<nb, 256, 0, h->stream>>>(N, rhs, dz, res, h->red);
    ++h->launches;
    k_final_sum<<<1, 256, 0, h->stream>>>(nb, h->red, h->red_out);
    ++h->launches;
    KQ_CUDA(h, cudaMemcpyAsync(h->h_red, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    KQ_CUDA(h, cudaStreamSynchronize(h->stream));
    resn = sqrt(h->h_red[0]);
    if (!(resn <= 0.5 * bn)) {
      cold = true;   // the old direction does not help (or is not finite)
      resn = bn;
    } else if (resn <= o.tol * bn) {
      s.rel_res = resn / bn;
      if (st) *st = s;
      return KQ_OK;
    }
  }
  if (cold) {
    KQ_CUDA(h, cudaMemsetAsync(z, 0, N * sizeof(double), h->stream));
    KQ_CUDA(h, cudaMemcpyAsync(res, rhs, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  }
  int total = 0;
  const int mixed = o.precision == KQ_PREC_MIXED;
  const int max_passes = (mixed ? o.refine_steps : 0) + 3;
  kq_status rc = KQ_OK;
  // up to refine_steps FP32 correction passes, each restarted from the true
  // (FP64) residual, then FP64 passes
  for (int pass = 0; pass < max_passes; ++pass) {
    const int prec = (mixed && pass < o.refine_steps) ? KQ_PREC_MIXED : KQ_PREC_F64;
    double rel = o.tol * bn / resn;
    if (prec == KQ_PREC_MIXED) rel = std::max(rel, o.inner_tol);
    rel = std::min(rel, 0.5);
    const int budget = o.maxit - total;
    if (budget <= 0) break;
    int it = 0;
    h->lz_on = h->record && pass == 0;
    rc = launch(h, prec, res, dz, rel, budget, 0, &it, nullptr, nullptr);
    if (h->lz_on) {
      h->lz_on = false;
      lanczos_extremes(h, it);
    }
    s.kernel_ms += h->last_kernel_ms;
    total += it;
    // products inside the launch: one per iteration
    const int prods = it;
    s.products += prods + 1;   // and the FP64 residual product below
    if (prec == KQ_PREC_F64) {
      s.iters_f64 += it;
      s.products_f64 += prods;
      s.kernel_ms_f64 += h->last_kernel_ms;
      s.launches_f64 += 1;
    }
    s.passes++;
    if (rc != KQ_OK) break;
    k_add<<<256, 256, 0, h->stream>>>(N, z, dz);
    ++h->launches;
    float ms = 0.f;
    rc = pcg_apply(h, z, dz, KQ_PREC_F64, &ms);
    s.kernel_ms += ms;
    s.kernel_ms_f64 += ms;
    s.products_f64 += 1;
    s.launches_f64 += 1;
    if (rc != KQ_OK) break;
    const int nb = 256;
    k_axpy_res<<<nb, 256, 0, h->stream>>>(N, rhs, dz, res, h->red);
    ++h->launches;
    k_final_sum<<<1, 256, 0, h->stream>>>(nb, h->red, h->red_out);
    ++h->launches;
    KQ_CUDA(h, cudaMemcpyAsync(h->h_red, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    KQ_CUDA(h, cudaStreamSynchronize(h->stream));
    resn = sqrt(h->h_red[0]);
    if (!(resn == resn)) { rc = kq_fail(h, KQ_ERR_NUMERIC, "PCG residual is NaN"); break; }
    if (resn <= o.tol * bn) break;
    if (total >= o.maxit) break;
  }
  s.iters = total;
  s.rel_res = resn / bn;
  if (rc == KQ_OK && resn > o.tol * bn) rc = KQ_WARN_PCG_MAXIT;
  s.status = rc;
  if (st) *st = s;
  return rc;
}

// ---------------------------------------------------------------- batched solver, captured graph
// The lock-step IPM iteration of the batch is captured once in a CUDA graph
// (batch.cu) and replayed; every decision the host made between launches is
// taken on the device from per-QP control words (QpCtl): which precision a
// correction pass runs in, when a Newton solve stops, the step lengths, the
// mu rule and when a QP is done.  Three argument arrays live on the device
// (FP32 solve, FP64 solve, FP64 apply), built before capture; the control
// kernels only switch problems on and off and set their tolerances.
namespace {

__device__ __forceinline__ PcgArgs *gargs_of(unsigned char *g, int which, int nq) {
  return reinterpret_cast<PcgArgs *>(g) + (size_t)which * nq;
}

__global__ void k_gctl_pcg_init(QpCtl *ctl, int nq, int mixed) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    QpCtl &c = ctl[q];
    c.pcg_done = c.active ? 0 : 1;
    if (c.used > 0) c.w_prev = c.used;
    c.used = 0;
    c.fp32_ok = mixed && c.f32_pays;
    c.resn = 0.0;
    c.bnorm = 0.0;
    c.ran = 0;
  }
}

// pass setup: precision and relative tolerance of this correction pass
__global__ void k_gctl_pass_setup(QpCtl *ctl, unsigned char *g, int nq, int pass, double tol,
                                  double inner_tol, int maxit, int refine_steps) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    QpCtl &c = ctl[q];
    PcgArgs *a32 = gargs_of(g, 0, nq) + q, *a64 = gargs_of(g, 1, nq) + q, *aap = gargs_of(g, 2, nq) + q;
    int run = c.active && !c.pcg_done;
    if (run && maxit - c.used <= 0) { c.pcg_done = 1; run = 0; }
    const int prec = (c.fp32_ok && pass < refine_steps) ? KQ_PREC_MIXED : KQ_PREC_F64;
    double rel = pass == 0 ? tol : tol * c.bnorm / fmax(c.resn, 1e-300);
    if (prec == KQ_PREC_MIXED) rel = fmax(rel, inner_tol);
    rel = fmin(rel, 0.5);
    PcgArgs *as = prec == KQ_PREC_MIXED ? a32 : a64;
    as->tol2 = rel * rel;
    as->maxit = maxit - c.used;
    a32->run = run && prec == KQ_PREC_MIXED;
    a64->run = run && prec == KQ_PREC_F64;
    aap->run = run;
    c.ran = run;
    c.prec = prec;
    c.resn_before = c.resn;
    c.tol_rel = tol;
  }
}

// pass finish: iterations, the true residual |rhs - K z| (reduced by the
// handle's kernels into redout[q][8]), the FP32 rule, stop or continue
__global__ void k_gctl_pass_finish(QpCtl *ctl, const int *iters, const int *errs, const double *resn,
                                   double *const *redout, int nq, int pass, int last, int maxit) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    QpCtl &c = ctl[q];
    if (!c.ran) continue;
    const int reg = c.prec == KQ_PREC_MIXED ? 0 : 1;
    const int e = errs[reg * nq + q] ? errs[reg * nq + q] : errs[2 * nq + q];
    if (e) {
      c.status = e == 7 ? KQ_ERR_TIMEOUT : (e == 4 ? KQ_ERR_NOT_CONVEX : KQ_ERR_NUMERIC);
      c.active = 0;
      c.pcg_done = 1;
      continue;
    }
    const int its = iters[reg * nq + q];
    if (pass == 0) c.bnorm = sqrt(resn[2 * (reg * nq + q) + 1]);
    c.used += its;
    c.pcg_iters += its;
    const double rn = sqrt(redout[q][8]);
    if (!(rn == rn)) {
      c.status = KQ_ERR_NUMERIC;
      c.active = 0;
      c.pcg_done = 1;
      continue;
    }
    c.resn = rn;
    if (c.prec == KQ_PREC_MIXED && pass > 0 && rn > 0.5 * c.resn_before) c.fp32_ok = 0;
    if (c.prec == KQ_PREC_MIXED && pass == 0 && rn > 0.5 * c.bnorm) c.fp32_ok = 0;
    if (rn <= c.tol_rel * c.bnorm || c.bnorm == 0.0) {
      c.pcg_done = 1;
    } else if (c.used >= maxit) {
      c.pcg_done = 1;
      c.maxit_hits++;
    } else if (last) {
      c.maxit_hits++;   // passes used up with the tolerance not met; the step is taken
    }
  }
}

// step lengths of Eq. (10) from the ratio-test minima (redout[q][4..5])
__global__ void k_gctl_step(QpCtl *ctl, double *const *redout, int nq, double gamma) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    QpCtl &c = ctl[q];
    if (!c.active) continue;
    c.ax = fmin(1.0, gamma * redout[q][4]);
    c.al = fmin(1.0, gamma * redout[q][5]);
    if (!(c.ax == c.ax) || !(c.al == c.al)) {
      c.status = KQ_ERR_NUMERIC;
      c.active = 0;
    }
  }
}

// the mu rule of Algorithm 1 from |r|^2 (redout[q][10..14]): return when
// |r| < mu and mu < mu_tol, else divide mu by 10 when |r| < mu
__global__ void k_gctl_mu_rule(QpCtl *ctl, double *const *redout, int nq, double mu0, double mu_tol) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    QpCtl &c = ctl[q];
    if (!c.active) continue;
    const double *r = redout[q] + 10;
    const double rn = sqrt(r[0] + r[1] + r[2] + r[3] + r[4]);
    c.ipm_iters++;
    if (!(rn == rn)) {
      c.status = KQ_ERR_NUMERIC;
      c.active = 0;
      continue;
    }
    if (rn < c.mu) {
      if (c.mu < mu_tol) {
        c.active = 0;
        c.status = KQ_OK;
      } else {
        c.kexp++;
        c.mu = mu0 * pow(10.0, -(double)c.kexp);
      }
    }
  }
}

__global__ void k_gctl_count(const QpCtl *ctl, int nq, int *count) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int c = 0;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) c += ctl[q].active;
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) *count = s;
}

// The team plan of one correction pass made on the device (the captured
// graph's counterpart of plan_teams, same rule): over the QPs that run in
// this pass (ctl.ran), costed by their cost per product times the iterations
// of their previous Newton solve, a QP worth two or more CTAs gets a team of
// that size (capped, shrunk to the room left); the rest are packed onto
// single-CTA teams, costliest first onto the least-loaded one.  One CTA of
// 1024 threads.  Writes cta_team (-1: idle CTA), teams, team_qps, the team
// size of every running QP into its three argument records, and zeroes the
// grid-barrier counters of the running QPs (team sizes change between passes;
// the barrier needs a counter that is a multiple of the team size).
constexpr int KQ_SCHED_MAX_Q = 2048;

size_t schedule_smem(int nq, int G) {
  return (size_t)(nq + G) * sizeof(double) + (size_t)(2 * nq + G + 1) * sizeof(int);
}

__global__ void __launch_bounds__(1024) k_gctl_schedule(const QpCtl *__restrict__ ctl, unsigned char *g,
                                                       int nq, int G, const double *__restrict__ q_cost,
                                                       const int *__restrict__ q_cap, int *cta_team,
                                                       TeamInfo *teams, int *team_qps) {
  extern __shared__ __align__(16) unsigned char sm[];
  double *cost = reinterpret_cast<double *>(sm);     // nq: cost of a running QP, -1 otherwise
  double *load = cost + nq;                          // G: load of each single-CTA team
  int *order = reinterpret_cast<int *>(load + G);    // k: running QPs, costliest first
  int *bin = order + nq;                             // single-CTA team of order[i]
  int *off = bin + nq;                               // G + 1: member offsets of those teams
  __shared__ double s_red[64];
  __shared__ double s_total;
  __shared__ int s_k, s_qpos, s_used, s_nsingle;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  double v[2] = {0.0, 0.0};   // total cost, running QPs
  for (int q = tid; q < nq; q += nt) {
    const QpCtl &c = ctl[q];
    const double w = c.ran ? q_cost[q] * (double)max(1, c.w_prev) : -1.0;
    cost[q] = w;
    if (c.ran) { v[0] += w; v[1] += 1.0; }
  }
  block_sum<2>(v, s_red);
  if (tid == 0) { s_total = v[0]; s_k = (int)(v[1] + 0.5); }
  __syncthreads();
  const double total = s_total;
  const int k = s_k;
  // rank of every running QP: costlier first, ties to the lower index
  for (int q = tid; q < nq; q += nt) {
    const double cq = cost[q];
    if (cq < 0.0) continue;
    int r = 0;
    for (int p = 0; p < nq; ++p) {
      const double cp = cost[p];
      r += (cp > cq) || (cp == cq && p < q);
    }
    order[r] = q;
  }
  __syncthreads();
  // teams of two or more CTAs (sequential: each takes from the room left)
  if (tid == 0) {
    int used = 0, i = 0;
    for (; i < k; ++i) {
      const int j = order[i];
      int t = (int)floor((double)G * cost[j] / total);
      t = min(t, q_cap[j]);
      const int room = (i + 1 < k) ? G - 1 - used : G - used;
      t = min(t, room);
      if (t < 2) break;
      teams[i] = TeamInfo{used, t, i, i + 1};
      team_qps[i] = j;
      used += t;
    }
    s_qpos = i;
    s_used = used;
    s_nsingle = (i < k) ? max(1, G - used) : 0;
  }
  __syncthreads();
  const int qpos = s_qpos, used = s_used, nsingle = s_nsingle;
  for (int c = tid; c < nsingle; c += nt) load[c] = 0.0;
  __syncthreads();
  // the rest onto single-CTA teams: costliest first onto the least-loaded
  // team (ties to the lower team), one warp
  if (tid < 32) {
    for (int i = qpos; i < k; ++i) {
      double best = INFINITY;
      int bi = 0x7fffffff;
      for (int c = lane; c < nsingle; c += 32) {
        const double l = load[c];
        if (l < best) { best = l; bi = c; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        load[bi] += cost[order[i]];
        bin[i] = bi;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int c = 0; c <= nsingle; ++c) off[c] = 0;
    for (int i = qpos; i < k; ++i) off[bin[i] + 1]++;
    for (int c = 0; c < nsingle; ++c) off[c + 1] += off[c];
    for (int c = 0; c < nsingle; ++c)
      teams[qpos + c] = TeamInfo{used + c, 1, qpos + off[c], qpos + off[c + 1]};
    for (int i = qpos; i < k; ++i) team_qps[qpos + off[bin[i]]++] = order[i];
  }
  __syncthreads();
  for (int x = tid; x < G; x += nt) {
    int t = -1;
    if (x >= used) {
      if (x < used + nsingle) t = qpos + (x - used);
    } else {
      for (int i = 0; i < qpos; ++i)
        if (x >= teams[i].first_cta && x < teams[i].first_cta + teams[i].size) { t = i; break; }
    }
    cta_team[x] = t;
  }
  for (int i = tid; i < k; i += nt) {
    const int j = order[i];
    const unsigned size = i < qpos ? (unsigned)teams[i].size : 1u;
    for (int w = 0; w < 3; ++w) gargs_of(g, w, nq)[j].bar.nblocks = size;
    const PcgArgs &a = gargs_of(g, 0, nq)[j];
    *a.bar.count = 0u;
    *a.bar.gen = 0u;
  }
}

// which: 0 = the correction pass (each problem in its own precision), 2 = FP64 apply
template <class HS, class AS>
const void *batch_kernel_of(int which) {
  return which == 0 ? (const void *)pcg_batch_kernel_dual<HS, AS>
                    : (const void *)pcg_batch_kernel<HS, AS, double>;
}

const void *graph_kernel(const kq_problem *h0, int which) {
  if (h0->P.hdtype == KQ_BF16 && h0->P.adtype == KQ_F32) return batch_kernel_of<__nv_bfloat16, float>(which);
  if (h0->P.hdtype == KQ_F64 && h0->P.adtype == KQ_F64) return batch_kernel_of<double, double>(which);
  return nullptr;
}

}  // namespace

kq_status batch_graph_prepare(BatchPcg &B, const std::vector<kq_problem *> &hs,
                              const std::vector<double> &weight, std::string &err) {
  const int nq = (int)hs.size();
  if (!B.gargs) {
    B.gargs = balloc<unsigned char>(B.allocs, 3 * (size_t)nq * sizeof(PcgArgs));
    B.ctl = balloc<QpCtl>(B.allocs, nq);
    B.redout = balloc<double *>(B.allocs, nq);
    B.g_iters = balloc<int>(B.allocs, 3 * (size_t)nq);
    B.g_err = balloc<int>(B.allocs, 3 * (size_t)nq);
    B.g_resn = balloc<double>(B.allocs, 6 * (size_t)nq);
    B.d_count = balloc<int>(B.allocs, 1);
    B.q_cost = balloc<double>(B.allocs, nq);
    B.q_cap = balloc<int>(B.allocs, nq);
    if (!B.gargs || !B.ctl || !B.redout || !B.g_iters || !B.g_err || !B.g_resn || !B.d_count ||
        !B.q_cost || !B.q_cap) {
      err = "batch graph work space";
      return KQ_ERR_OOM;
    }
    if (cudaMallocHost((void **)&B.h_count, sizeof(int)) != cudaSuccess) {
      err = "batch graph pinned count";
      return KQ_ERR_OOM;
    }
    std::vector<double *> ro(nq);
    for (int q = 0; q < nq; ++q) ro[q] = hs[q]->red_out;
    if (cudaMemcpy(B.redout, ro.data(), nq * sizeof(double *), cudaMemcpyHostToDevice) != cudaSuccess) {
      err = "batch graph pointers";
      return KQ_ERR_CUDA;
    }
  }
  // per-QP cost and team cap for the device-side plan (a batch of more than
  // KQ_SCHED_MAX_Q QPs keeps the plan made here for the whole capture)
  {
    std::vector<double> qc(nq);
    std::vector<int> qk(nq);
    for (int q = 0; q < nq; ++q) {
      qc[q] = unit_cost(hs[q], &B.tune);
      qk[q] = team_cap(hs[q], &B.tune);
    }
    if (cudaMemcpy(B.q_cost, qc.data(), nq * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B.q_cap, qk.data(), nq * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
      err = "batch graph costs";
      return KQ_ERR_CUDA;
    }
    B.dev_sched = nq <= KQ_SCHED_MAX_Q;
  }
  // teams over the problems still iterating (weight > 0)
  std::vector<int> idx;
  std::vector<double> w;
  for (int q = 0; q < nq; ++q)
    if (weight[q] > 0.0) { idx.push_back(q); w.push_back(weight[q]); }
  TeamPlan tp;
  if (!idx.empty()) tp = plan_teams(B.G, hs, idx, &w, &B.tune);
  std::vector<int> team_size(nq, 1);
  for (size_t j = 0; j < idx.size(); ++j) team_size[idx[j]] = tp.teams[tp.team_of[j]].size;
  for (int &j : tp.team_qps) j = idx[j];          // list positions -> problem indices
  std::vector<PcgArgs> args(3 * (size_t)nq);
  size_t smem[3] = {0, 0, 0};
  for (int which = 0; which < 3; ++which) {
    for (int q = 0; q < nq; ++q) {
      kq_problem *h = hs[q];
      PcgWork &W = h->W;
      PcgArgs &a = args[(size_t)which * nq + q];
      a = PcgArgs{};
      a.P = h->P;
      a.Dl = h->K.Dl; a.Du = h->K.Du; a.cl = h->K.cl; a.cu = h->K.cu;
      a.dg = h->K.dg; a.diag = h->K.diag; a.mu = h->K.mu;
      a.apply = which == 2;
      a.rhs = a.apply ? h->z : h->tmp;
      a.z = h->zref;
      a.r = W.r; a.y = W.y; a.pb0 = W.pb0; a.pb1 = W.pb1; a.qlam = W.qlam;
      a.accx = which == 0 ? (void *)W.accx32 : (void *)W.accx64;
      a.g = nullptr; a.slots = W.slots;
      a.win_cap = (int)((h->n + 7) & ~(int64_t)7);
      a.bar.count = W.bar; a.bar.gen = W.bar + 1; a.bar.err = B.g_err + (size_t)which * nq + q;
      a.bar.nblocks = (unsigned)team_size[q];
      a.bar.budget_ns = (uint64_t)(h->timeout_s * 1e9);
      a.tol2 = 0.0; a.maxit = 0;
      a.iters = B.g_iters + (size_t)which * nq + q;
      a.resn = B.g_resn + 2 * ((size_t)which * nq + q);
      a.stages = 2; a.producer = 0; a.copy_piece = 16;
      a.stag_window = which == 0 ? W.stag_window : 0;
      a.coefA = W.coefA;
      a.dinv = W.dinv;
      a.run = 0;
      a.colpass_min_n = B.tune.colpass_min_n;
      if (weight[q] > 0.0)
        smem[which] = std::max(smem[which], (size_t)2 * a.win_cap * (which == 0 ? sizeof(float) : sizeof(double)));
    }
  }
  cudaError_t e;
  if ((e = cudaMemcpy(B.gargs, args.data(), args.size() * sizeof(PcgArgs), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(B.g_err, 0, 3 * (size_t)nq * sizeof(int))) != cudaSuccess) {
    err = std::string("batch graph arguments: ") + cudaGetErrorString(e);
    return KQ_ERR_CUDA;
  }
  // grid-barrier counters start at zero; within one capture every launch of
  // a problem uses the same team size, so the counter stays a multiple of it
  for (int q = 0; q < nq; ++q)
    if (cudaMemset(hs[q]->W.bar, 0, 2 * sizeof(unsigned int)) != cudaSuccess) {
      err = "batch graph barrier reset";
      return KQ_ERR_CUDA;
    }
  // a device-planned launch covers every CTA; the plan leaves some idle
  B.gblocks = (B.dev_sched && tp.nblocks > 0) ? B.G : tp.nblocks;
  if (B.gblocks > 0) {
    if ((e = cudaMemcpy(B.cta_team, tp.cta_team.data(), tp.nblocks * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(B.teams, tp.teams.data(), tp.teams.size() * sizeof(TeamInfo), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(B.team_qps, tp.team_qps.data(), tp.team_qps.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) {
      err = std::string("batch graph teams: ") + cudaGetErrorString(e);
      return KQ_ERR_CUDA;
    }
    smem[0] = std::max(smem[0], smem[1]);   // the pass launch runs either precision
    for (int which : {0, 2}) {
      const void *f = graph_kernel(hs[0], which);
      if (!f) { err = "batched PCG supports bf16 H with f32 A, or f64 H with f64 A"; return KQ_ERR_ARG; }
      B.gsmem[which] = std::max<size_t>(smem[which], 16);
      int per_sm = 0;
      if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.gsmem[which]) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 512, B.gsmem[which]) != cudaSuccess ||
          per_sm * B.G < B.gblocks) {
        err = "batched PCG grid does not fit";
        return KQ_ERR_ARG;
      }
    }
  }
  return KQ_OK;
}

// one batched launch of kind `which` (0: the correction pass, each problem in
// its own precision; 2: FP64 apply) as a cooperative launch that stream
// capture records as a graph node
kq_status batch_graph_launch(BatchPcg &B, const kq_problem *h0, int which, cudaStream_t s,
                             std::string &err) {
  if (B.gblocks == 0) return KQ_OK;
  const void *f = graph_kernel(h0, which);
  PcgArgs *pa = reinterpret_cast<PcgArgs *>(B.gargs) + (size_t)which * B.nqp;
  PcgArgs *p64 = reinterpret_cast<PcgArgs *>(B.gargs) + (size_t)B.nqp;
  const TeamInfo *pt = reinterpret_cast<const TeamInfo *>(B.teams);
  void *kargs_pass[] = {(void *)&pa, (void *)&p64, (void *)&B.cta_team, (void *)&pt, (void *)&B.team_qps};
  void *kargs_one[] = {(void *)&pa, (void *)&B.cta_team, (void *)&pt, (void *)&B.team_qps};
  void **kargs = which == 0 ? kargs_pass : kargs_one;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(B.gblocks);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = B.gsmem[which];
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelExC(&cfg, f, kargs);
  if (e != cudaSuccess) {
    err = std::string("batch graph launch: ") + cudaGetErrorString(e);
    return KQ_ERR_CUDA;
  }
  B.launches++;
  return KQ_OK;
}

void batch_graph_pcg_init(BatchPcg &B, int mixed, cudaStream_t s) {
  k_gctl_pcg_init<<<(B.nqp + 255) / 256, 256, 0, s>>>(B.ctl, B.nqp, mixed);
}
void batch_graph_pass_setup(BatchPcg &B, int pass, const kq_pcg_opts &o, cudaStream_t s) {
  k_gctl_pass_setup<<<(B.nqp + 255) / 256, 256, 0, s>>>(B.ctl, B.gargs, B.nqp, pass, o.tol, o.inner_tol,
                                                        o.maxit, o.precision == KQ_PREC_MIXED ? o.refine_steps : 0);
}
void batch_graph_schedule(BatchPcg &B, cudaStream_t s) {
  if (!B.dev_sched || B.gblocks == 0) return;
  k_gctl_schedule<<<1, 1024, schedule_smem(B.nqp, B.G), s>>>(
      B.ctl, B.gargs, B.nqp, B.G, B.q_cost, B.q_cap, B.cta_team,
      reinterpret_cast<TeamInfo *>(B.teams), B.team_qps);
}
void batch_graph_pass_finish(BatchPcg &B, int pass, int last, int maxit, cudaStream_t s) {
  k_gctl_pass_finish<<<(B.nqp + 255) / 256, 256, 0, s>>>(B.ctl, B.g_iters, B.g_err, B.g_resn, B.redout,
                                                         B.nqp, pass, last, maxit);
}
void batch_graph_step(BatchPcg &B, double gamma, cudaStream_t s) {
  k_gctl_step<<<(B.nqp + 255) / 256, 256, 0, s>>>(B.ctl, B.redout, B.nqp, gamma);
}
void batch_graph_mu_rule(BatchPcg &B, double mu0, double mu_tol, cudaStream_t s) {
  k_gctl_mu_rule<<<(B.nqp + 255) / 256, 256, 0, s>>>(B.ctl, B.redout, B.nqp, mu0, mu_tol);
}
void batch_graph_count(BatchPcg &B, cudaStream_t s) {
  k_gctl_count<<<1, 256, 0, s>>>(B.ctl, B.nqp, B.d_count);
  cudaMemcpyAsync(B.h_count, B.d_count, sizeof(int), cudaMemcpyDeviceToHost, s);
}
