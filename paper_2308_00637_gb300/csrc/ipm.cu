// Interior point iteration (Algorithm 1) and the C ABI.
//
// Per iteration, on the device in FP64:
//   1. residuals of Eq. (3) / right-hand side of Eq. (7) at (x, s, lam, mu),
//      the 2x2 reduction of Eq. (8) (D, dg, r1, r2) and the doubly augmented
//      right-hand side [r1 + 2B'D^-1 r2; r2] of Eq. (9), plus diag(K);
//   2. Jacobi-PCG solve of Eq. (9) (pcg.cu);
//   3. slack and bound-multiplier directions from the linearised Eq. (3);
//   4. ratio test, Eq. (10), as two min-reductions; update;
//   5. residual norm and the mu rule of section 3.2.
// Only the scalars (|r|, alpha_x, alpha_lam, PCG status) cross to the host.
#include "common.cuh"
#include "kq_internal.h"
#include <chrono>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

// batched solver's captured graph: a kernel of a QP that has stopped iterating returns at once
#define KQ_GATE(P) \
  if ((P).gate && *(P).gate == 0) return
constexpr int NB = 256;      // blocks of the grid-stride IPM kernels
constexpr int NT = 256;
thread_local std::string g_global_err;

// ---------------------------------------------------------------- create-time kernels
__global__ void k_flags(int64_t N, const double *lo, const double *hi, uint8_t *hl, uint8_t *hu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    hl[i] = isfinite(lo[i]) ? 1 : 0;
    hu[i] = isfinite(hi[i]) ? 1 : 0;
  }
}

// per-block min of v and min of -v (max) into part[b], part[NB + b]
__global__ void k_minmax(int64_t N, const double *v, double *part) {
  __shared__ double sh[32];
  double mn = INFINITY, mx = INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    mn = fmin(mn, v[i]);
    mx = fmin(mx, -v[i]);
  }
  mn = block_min(mn, sh);
  mx = block_min(mx, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = mn; part[NB + blockIdx.x] = mx; }
}

// qp_update: bounds replaced by unscaled values (new_l / new_u) are divided
// by their row norms; flags are recomputed from finiteness (scaling keeps it)
__global__ void k_flags_scaled(int64_t m, double *lA, double *uA, bool new_l, bool new_u,
                               const double *rho, uint8_t *hl, uint8_t *hu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (new_l) lA[i] *= rho[i];
    if (new_u) uA[i] *= rho[i];
    hl[i] = isfinite(lA[i]) ? 1 : 0;
    hu[i] = isfinite(uA[i]) ? 1 : 0;
  }
}

template <class HS>
__global__ void k_dense_diag(int64_t n, int64_t ld, const HS *H, double *d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = ld_as_f64(H, i * ld + i);
}

// Gaussian-kernel SVM Hessian (Eq. (6)), formed once:
// H_ij = y_i y_j exp(-gamma sum_k (X_ik - X_jk)^2) into the padded dense
// storage (row stride ld).  One 32 x 32 tile of H per CTA of 32 x 8 threads
// (four entries a thread); 32-feature slabs of the tile's two row blocks of X
// staged in shared memory; squared differences summed in FP64 in feature
// order, so H is exactly symmetric and its diagonal is y_i^2.
template <class HS>
__global__ void __launch_bounds__(256) k_rbf_build(int64_t n, int64_t d, const double *X,
                                                   const double *y, double gamma, int64_t ld,
                                                   HS *H) {
  __shared__ double xi[32][33], xj[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k0 = 0; k0 < d; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int64_t k = k0 + tx;
      xi[r][tx] = (i0 + r < n && k < d) ? X[(i0 + r) * d + k] : 0.0;
      xj[r][tx] = (j0 + r < n && k < d) ? X[(j0 + r) * d + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      const double b = xj[tx][k];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double t = xi[ty + 8 * u][k] - b;
        acc[u] = fma(t, t, acc[u]);
      }
    }
    __syncthreads();
  }
  const int64_t j = j0 + tx;
  if (j >= n) return;
  const double yj = y ? y[j] : 1.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + ty + 8 * u;
    if (i < n) st_from_f64(H, i * ld + j, (y ? y[i] : 1.0) * yj * exp(-gamma * acc[u]));
  }
}

// diag(Z diag(zw) Z' + diag(d0))_i = sum_c zw_c Z_ic^2 + d0_i (zw, d0 optional)
template <class ZS>
__global__ void k_rownorm2(int64_t rows, int64_t k, const ZS *Z, const double *zw,
                           const double *d0, double *d) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < rows; i += W) {
    double s = 0.0;
    for (int64_t c = lane; c < k; c += 32) {
      const double v = ld_as_f64(Z, i * k + c);
      s += (zw ? zw[c] : 1.0) * v * v;
    }
    s = warp_sum(s);
    if (lane == 0) d[i] = s + (d0 ? d0[i] : 0.0);
  }
}

// diag(2 P'WP)_j = sum_r 2 w_r P_rj^2
__global__ void k_csr_diag(int64_t nP, const int64_t *rowptr, const int32_t *col, const float *val,
                           const double *w, double scale, double *d) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < nP; r += W) {
    const double wr = scale * w[r];
    for (int64_t k = rowptr[r] + lane; k < rowptr[r + 1]; k += 32) {
      const double v = val[k];
      atomicAdd(d + col[k], wr * v * v);
    }
  }
}

// 1/||row||_2 of dense rows (or of the P rows selected by `rows`)
template <class AS>
__global__ void k_rho_dense(int64_t m, int64_t n, int64_t ld, const AS *A, double *rho) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < m; i += W) {
    double s = 0.0;
    for (int64_t c = lane; c < n; c += 32) { const double v = ld_as_f64(A, i * ld + c); s += v * v; }
    s = warp_sum(s);
    if (lane == 0) rho[i] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
  }
}

__global__ void k_rho_rows(int64_t m, const int32_t *rows, const int64_t *rowptr, const float *val,
                           double *rho) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < m; i += W) {
    const int64_t r = rows[i];
    double s = 0.0;
    for (int64_t k = rowptr[r] + lane; k < rowptr[r + 1]; k += 32) { const double v = val[k]; s += v * v; }
    s = warp_sum(s);
    if (lane == 0) rho[i] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
  }
}

// 1/||row||_2 of the rows of a CSR A
template <class AS>
__global__ void k_rho_acsr(int64_t m, const int64_t *rowptr, const AS *val, double *rho) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < m; i += W) {
    double s = 0.0;
    for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) { const double v = ld_as_f64(val, k); s += v * v; }
    s = warp_sum(s);
    if (lane == 0) rho[i] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
  }
}

__global__ void k_scale_vec(int64_t N, double *v, const double *rho, double sc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= rho ? rho[i] : sc;
}

__global__ void k_scale_rows(int64_t m, int64_t n, double *C, double *b, double *rhoC) {
  // one block per row: rho = 1/||C_e||, C_e *= rho, b_e *= rho
  __shared__ double sh[32];
  const int64_t e = blockIdx.x;
  double s[1] = {0.0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s[0] += C[e * n + j] * C[e * n + j];
  block_sum<1>(s, sh);
  __shared__ double rho;
  if (threadIdx.x == 0) { rho = s[0] > 0.0 ? 1.0 / sqrt(s[0]) : 1.0; rhoC[e] = rho; b[e] *= rho; }
  __syncthreads();
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) C[e * n + j] *= rho;
}

// max |v_i| per block; a NaN or an infinity gives +inf (fmax alone would drop NaN)
__global__ void k_max_abs(int64_t N, const double *v, double *part) {
  __shared__ double sh[32];
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(v[i]);
    mx = (a <= 1.79e308) ? fmax(mx, a) : INFINITY;
  }
  mx = -block_min(-mx, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = mx;
}

// CSR structure check: rowptr non-decreasing from 0 to nnz, 0 <= col < n,
// and (for ROWS_OF_P) 0 <= rows[i] < nP strictly increasing.  Sets *bad.
__global__ void k_check_csr(int64_t nP, int64_t n, int64_t nnz, const int64_t *rowptr,
                            const int32_t *col, int64_t m, const int32_t *rows, int *bad) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = tid; r < nP; r += stride) {
    if (rowptr[r] > rowptr[r + 1]) atomicOr(bad, 1);
  }
  if (tid == 0 && (rowptr[0] != 0 || rowptr[nP] != nnz)) atomicOr(bad, 1);
  for (int64_t k = tid; k < nnz; k += stride) {
    const int32_t c = col[k];
    if (c < 0 || c >= n) atomicOr(bad, 2);
  }
  for (int64_t i = tid; i < m; i += stride) {
    const int32_t r = rows[i];
    if (r < 0 || r >= nP || (i > 0 && rows[i - 1] >= r)) atomicOr(bad, 4);
  }
}

__global__ void k_prow2a(int64_t m, const int32_t *rows, int32_t *prow2a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    prow2a[rows[i]] = (int32_t)i;
}

// ---------------------------------------------------------------- initial point
__global__ void k_init_x(DevProb P, DevState S) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool fl = P.haslx[i], fu = P.hasux[i];
    double x = 0.0;
    if (fl && fu) x = 0.5 * (P.lx[i] + P.ux[i]);
    else if (fl) x = P.lx[i] + 1.0;
    else if (fu) x = P.ux[i] - 1.0;
    S.x[i] = x;
    S.slx[i] = fl ? fmax(x - P.lx[i], 1.0) : 1.0;
    S.sux[i] = fu ? fmax(P.ux[i] - x, 1.0) : 1.0;
    S.llx[i] = fl ? 1.0 : 0.0;
    S.lux[i] = fu ? 1.0 : 0.0;
  }
}

__global__ void k_init_rows(DevProb P, DevState S, const double *t) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.m; a += (int64_t)gridDim.x * blockDim.x) {
    const bool hl = P.hasl[a], hu = P.hasu[a];
    S.sl[a] = hl ? fmax(t[a] - P.lA[a], 1.0) : 1.0;
    S.su[a] = hu ? fmax(P.uA[a] - t[a], 1.0) : 1.0;
    S.ll[a] = hl ? 1.0 : 0.0;
    S.lu[a] = hu ? 1.0 : 0.0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.me; e += (int64_t)gridDim.x * blockDim.x)
    S.le[e] = 0.0;
}

// ---------------------------------------------------------------- products used by the IPM step
// t_a = rho_a A_a v  (all general rows),  tC_e = C_e v
template <class AS>
__global__ void k_rowdot_dense(DevProb P, const double *v, double *t, double *tC) {
  KQ_GATE(P);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const AS *A = reinterpret_cast<const AS *>(P.Ad);
  for (int64_t i = w0; i < P.m + P.me; i += W) {
    double s = 0.0;
    if (i < P.m) {
      for (int64_t c = lane; c < P.n; c += 32) s += ld_as_f64(A, i * P.ald + c) * v[c];
      s = warp_sum(s);
      if (lane == 0) t[i] = P.rhoA[i] * s;
    } else {
      const int64_t e = i - P.m;
      for (int64_t c = lane; c < P.n; c += 32) s += P.Cd[e * P.n + c] * v[c];
      s = warp_sum(s);
      if (lane == 0) tC[e] = s;
    }
  }
}

__global__ void k_rowdot_prows(DevProb P, const double *v, double *t, double *tC) {
  KQ_GATE(P);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < P.m + P.me; i += W) {
    double s = 0.0;
    if (i < P.m) {
      const int64_t r = P.arows[i];
      for (int64_t k = P.rowptr[r] + lane; k < P.rowptr[r + 1]; k += 32) s += (double)P.val[k] * v[P.col[k]];
      s = warp_sum(s);
      if (lane == 0) t[i] = P.rhoA[i] * s;
    } else {
      const int64_t e = i - P.m;
      for (int64_t c = lane; c < P.n; c += 32) s += P.Cd[e * P.n + c] * v[c];
      s = warp_sum(s);
      if (lane == 0) tC[e] = s;
    }
  }
}

// t_a = rho_a A_a v for the rows of a CSR A, tC_e = C_e v
template <class AS>
__global__ void k_rowdot_acsr(DevProb P, const double *v, double *t, double *tC) {
  KQ_GATE(P);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const AS *val = reinterpret_cast<const AS *>(P.aval);
  for (int64_t i = w0; i < P.m + P.me; i += W) {
    double s = 0.0;
    if (i < P.m) {
      for (int64_t k = P.arowptr[i] + lane; k < P.arowptr[i + 1]; k += 32)
        s += ld_as_f64(val, k) * v[P.acol[k]];
      s = warp_sum(s);
      if (lane == 0) t[i] = P.rhoA[i] * s;
    } else {
      const int64_t e = i - P.m;
      for (int64_t c = lane; c < P.n; c += 32) s += P.Cd[e * P.n + c] * v[c];
      s = warp_sum(s);
      if (lane == 0) tC[e] = s;
    }
  }
}

// y = P v for every row of P
__global__ void k_csr_rowdot(DevProb P, const double *v, double *y) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < P.nP; r += W) {
    double s = 0.0;
    for (int64_t k = P.rowptr[r] + lane; k < P.rowptr[r + 1]; k += 32) s += (double)P.val[k] * v[P.col[k]];
    s = warp_sum(s);
    if (lane == 0) y[r] = s;
  }
}

// hx = sigma H v (DENSE)
template <class HS>
__global__ void k_hx_dense(DevProb P, const double *v, double *hx) {
  KQ_GATE(P);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const HS *H = reinterpret_cast<const HS *>(P.Hd);
  for (int64_t i = w0; i < P.n; i += W) {
    double s = 0.0;
    for (int64_t c = lane; c < P.n; c += 32) s += ld_as_f64(H, i * P.hld + c) * v[c];
    s = warp_sum(s);
    if (lane == 0) hx[i] = P.hscale * s;
  }
}

// g = Z' v (LOWRANK, atomics over row blocks)
template <class ZS>
__global__ void k_zt(DevProb P, const double *v, double *g) {
  const ZS *Z = reinterpret_cast<const ZS *>(P.Z);
  const int64_t rows_per = ceil_div64(P.n, gridDim.x);
  const int64_t r0 = blockIdx.x * rows_per, r1 = min(P.n, r0 + rows_per);
  for (int64_t c = threadIdx.x; c < P.k; c += blockDim.x) {
    double s = 0.0;
    for (int64_t i = r0; i < r1; ++i) s += ld_as_f64(Z, i * P.k + c) * v[i];
    atomicAdd(g + c, s);
  }
}

// hx = sigma (Z diag(zw) g + d0 v)
template <class ZS>
__global__ void k_zg(DevProb P, const double *g, const double *v, double *hx) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const ZS *Z = reinterpret_cast<const ZS *>(P.Z);
  for (int64_t i = w0; i < P.n; i += W) {
    double s = 0.0;
    for (int64_t c = lane; c < P.k; c += 32) s += ld_as_f64(Z, i * P.k + c) * g[c] * (P.zw ? P.zw[c] : 1.0);
    s = warp_sum(s);
    if (lane == 0) hx[i] = P.hscale * (s + (P.d0 ? P.d0[i] * v[i] : 0.0));
  }
}

// ---------------------------------------------------------------- residual pass, row part
// Per general row a (t = rho A_a x) and equality row e (tC = C_e x):
//   r_lA = t - s_l - l,  r_uA = -t - s_u + u,  r_c1 = lam_l s_l - mu,  r_c2 = lam_u s_u - mu
//   D_l = s_l / lam_l,   r2_l = -r_lA - r_c1 / lam_l   (and the same for u)
//   r_e = tC - b + mu lam_e,  D_e = mu,  r2_e = -r_e
// and the per-row coefficients of the three scatters (pre-multiplied by the
// row scale for general rows):
//   c1 (r_H):   -(lam_l - lam_u) ;  -lam_e
//   c2 (rhs):   2 (r2_l / D_l - r2_u / D_u) ;  2 r2_e / mu
//   c3 (diag):  2 (1/D_l + 1/D_u) ;  2 / mu          (multiplies the squared row)
struct RowCoef { double *c1, *c2, *c3; };

__global__ void k_rows_resid(DevProb P, DevState S, DevKKT K, const double *t, const double *tC,
                             RowCoef cf, double *part) {
  KQ_GATE(P);
  __shared__ double sh[32 * 2];
  const double mu = P.mu_dev ? *P.mu_dev : K.mu;
  double ss[2] = {0.0, 0.0};   // [primal (row and equality residuals), complementarity]
  const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.m; a += (int64_t)gridDim.x * blockDim.x) {
    const bool hl = P.hasl[a], hu = P.hasu[a];
    double c1 = 0.0, c2 = 0.0, c3 = 0.0;
    double rl = 0.0, ru = 0.0, r1 = 0.0, r2 = 0.0, Dl = 1.0, Du = 1.0, r2l = 0.0, r2u = 0.0;
    if (hl) {
      rl = t[a] - S.sl[a] - P.lA[a];
      r1 = S.ll[a] * S.sl[a] - mu;
      Dl = S.sl[a] / S.ll[a];
      r2l = -rl - r1 / S.ll[a];
      c1 -= S.ll[a];
      c2 += 2.0 * r2l / Dl;
      c3 += 2.0 / Dl;
    }
    if (hu) {
      ru = -t[a] - S.su[a] + P.uA[a];
      r2 = S.lu[a] * S.su[a] - mu;
      Du = S.su[a] / S.lu[a];
      r2u = -ru - r2 / S.lu[a];
      c1 += S.lu[a];
      c2 -= 2.0 * r2u / Du;
      c3 += 2.0 / Du;
    }
    const double rho = P.rhoA[a];
    cf.c1[a] = rho * c1;
    cf.c2[a] = rho * c2;
    cf.c3[a] = rho * rho * c3;
    K.rlA[a] = rl; K.ruA[a] = ru; K.rc1[a] = r1; K.rc2[a] = r2;
    K.Dl[a] = Dl; K.Du[a] = Du;
    K.cl[a] = hl ? 1.0 / Dl : 0.0;
    K.cu[a] = hu ? 1.0 / Du : 0.0;
    K.rhs[lo_off + a] = r2l;
    K.rhs[up_off + a] = r2u;
    K.diag[lo_off + a] = Dl;
    K.diag[up_off + a] = Du;
    ss[0] += rl * rl + ru * ru;
    ss[1] += r1 * r1 + r2 * r2;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.me; e += (int64_t)gridDim.x * blockDim.x) {
    const double re = tC[e] - P.b[e] + mu * S.le[e];
    K.re[e] = re;
    cf.c1[P.m + e] = -S.le[e];
    cf.c2[P.m + e] = 2.0 * (-re) / mu;
    cf.c3[P.m + e] = 2.0 / mu;
    K.rhs[P.n + e] = -re;
    K.diag[P.n + e] = mu;
    ss[0] += re * re;
  }
  block_sum<2>(ss, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = ss[0]; part[NB + blockIdx.x] = ss[1]; }
}

// scatter for dense rows (general rows of a dense A and the equality rows):
// thread per column j:  acc_k[j] = sum_rows c_k(row) * row_j (^2 for k = 3)
template <class AS>
__global__ void k_rows_scatter_dense(DevProb P, RowCoef cf, double *acc1, double *acc2, double *acc3) {
  KQ_GATE(P);
  const AS *A = reinterpret_cast<const AS *>(P.Ad);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.n; j += (int64_t)gridDim.x * blockDim.x) {
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (P.akind == KQ_A_DENSE) {
      for (int64_t a = 0; a < P.m; ++a) {
        const double v = ld_as_f64(A, a * P.ald + j);
        s1 += cf.c1[a] * v; s2 += cf.c2[a] * v; s3 += cf.c3[a] * v * v;
      }
    }
    for (int64_t e = 0; e < P.me; ++e) {
      const double v = P.Cd[e * P.n + j];
      s1 += cf.c1[P.m + e] * v; s2 += cf.c2[P.m + e] * v; s3 += cf.c3[P.m + e] * v * v;
    }
    acc1[j] += s1; acc2[j] += s2; acc3[j] += s3;
  }
}

// scatter through the rows of a CSR A: acc_k += A' c_k (k = 1, 2), acc3 += (A.^2)' c3
// (the coefficients already carry the row scale, c3 its square)
template <class AS>
__global__ void k_acsr_scatter(DevProb P, RowCoef cf, double *acc1, double *acc2, double *acc3) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const AS *val = reinterpret_cast<const AS *>(P.aval);
  for (int64_t a = w0; a < P.m; a += W) {
    const double u1 = cf.c1[a], u2 = cf.c2[a], u3 = cf.c3[a];
    if (u1 == 0.0 && u2 == 0.0 && u3 == 0.0) continue;
    for (int64_t k = P.arowptr[a] + lane; k < P.arowptr[a + 1]; k += 32) {
      const double v = ld_as_f64(val, k);
      const int c = P.acol[k];
      atomicAdd(acc1 + c, u1 * v);
      atomicAdd(acc2 + c, u2 * v);
      atomicAdd(acc3 + c, u3 * v * v);
    }
  }
}

// scatter through P: acc1 += P'(w2 y + c1), acc2 += P'c2, acc3 += (P.^2)'(w2 + c3)
__global__ void k_csr_scatter(DevProb P, const double *y, RowCoef cf, double *acc1, double *acc2, double *acc3) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < P.nP; r += W) {
    const int ai = P.prow2a[r];
    double u1 = y ? P.w2[r] * y[r] : 0.0, u2 = 0.0, u3 = P.w2[r];
    if (ai >= 0) { u1 += cf.c1[ai]; u2 += cf.c2[ai]; u3 += cf.c3[ai]; }
    for (int64_t k = P.rowptr[r] + lane; k < P.rowptr[r + 1]; k += 32) {
      const double v = P.val[k];
      const int c = P.col[k];
      atomicAdd(acc1 + c, u1 * v);
      if (u2 != 0.0) atomicAdd(acc2 + c, u2 * v);
      atomicAdd(acc3 + c, u3 * v * v);
    }
  }
}

// x part: r_H, bound residuals, r1, rhs_x = r1 + acc2, diag_x = hdiag + dg + acc3
__global__ void k_x_resid(DevProb P, DevState S, DevKKT K, const double *hx, const double *acc1,
                          const double *acc2, const double *acc3, double *part) {
  KQ_GATE(P);
  __shared__ double sh[32 * 3];
  const double mu = P.mu_dev ? *P.mu_dev : K.mu;
  double ss[3] = {0.0, 0.0, 0.0};   // [bound residuals, r_H, bound complementarity]
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool fl = P.haslx[i], fu = P.hasux[i];
    const double x = S.x[i];
    double rH = hx[i] + P.p[i] + acc1[i];
    double rlx = 0, rux = 0, rc3 = 0, rc4 = 0, dg = 0, r1 = 0;
    if (fl) { rH -= S.llx[i]; rlx = x - S.slx[i] - P.lx[i]; rc3 = S.llx[i] * S.slx[i] - mu; dg += S.llx[i] / S.slx[i]; }
    if (fu) { rH += S.lux[i]; rux = -x - S.sux[i] + P.ux[i]; rc4 = S.lux[i] * S.sux[i] - mu; dg += S.lux[i] / S.sux[i]; }
    r1 = -rH;
    if (fl) r1 += -rc3 / S.slx[i] - S.llx[i] / S.slx[i] * rlx;
    if (fu) r1 += rc4 / S.sux[i] + S.lux[i] / S.sux[i] * rux;
    K.rH[i] = rH; K.rlx[i] = rlx; K.rux[i] = rux; K.rc3[i] = rc3; K.rc4[i] = rc4; K.dg[i] = dg;
    K.rhs[i] = r1 + acc2[i];
    K.diag[i] = P.hdiag[i] + dg + acc3[i];
    ss[0] += rlx * rlx + rux * rux;
    ss[1] += rH * rH;
    ss[2] += rc3 * rc3 + rc4 * rc4;
  }
  block_sum<3>(ss, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = ss[0];
    part[NB + blockIdx.x] = ss[1];
    part[2 * NB + blockIdx.x] = ss[2];
  }
}

// ---------------------------------------------------------------- step recovery and ratio test
__global__ void k_recover_ratio(DevProb P, DevState S, DevKKT K, const double *z, const double *t,
                                double *dsl, double *dsu, double *dslx, double *dsux,
                                double *dllx, double *dlux, double *part) {
  KQ_GATE(P);
  __shared__ double sh[32];
  double ax = INFINITY, al = INFINITY;
  const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.m; a += (int64_t)gridDim.x * blockDim.x) {
    if (P.hasl[a]) {
      const double ds = t[a] + K.rlA[a], dl = z[lo_off + a];
      dsl[a] = ds;
      if (ds < 0.0) ax = fmin(ax, -S.sl[a] / ds);
      if (dl < 0.0) al = fmin(al, -S.ll[a] / dl);
    } else dsl[a] = 0.0;
    if (P.hasu[a]) {
      const double ds = -t[a] + K.ruA[a], dl = z[up_off + a];
      dsu[a] = ds;
      if (ds < 0.0) ax = fmin(ax, -S.su[a] / ds);
      if (dl < 0.0) al = fmin(al, -S.lu[a] / dl);
    } else dsu[a] = 0.0;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double dx = z[i];
    if (P.haslx[i]) {
      const double ds = dx + K.rlx[i];
      const double dl = -(K.rc3[i] + S.llx[i] * ds) / S.slx[i];
      dslx[i] = ds; dllx[i] = dl;
      if (ds < 0.0) ax = fmin(ax, -S.slx[i] / ds);
      if (dl < 0.0) al = fmin(al, -S.llx[i] / dl);
    } else { dslx[i] = 0.0; dllx[i] = 0.0; }
    if (P.hasux[i]) {
      const double ds = -dx + K.rux[i];
      const double dl = -(K.rc4[i] + S.lux[i] * ds) / S.sux[i];
      dsux[i] = ds; dlux[i] = dl;
      if (ds < 0.0) ax = fmin(ax, -S.sux[i] / ds);
      if (dl < 0.0) al = fmin(al, -S.lux[i] / dl);
    } else { dsux[i] = 0.0; dlux[i] = 0.0; }
  }
  ax = block_min(ax, sh);
  al = block_min(al, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = ax; part[NB + blockIdx.x] = al; }
}

__global__ void k_update(DevProb P, DevState S, const double *z, const double *dsl, const double *dsu,
                         const double *dslx, const double *dsux, const double *dllx,
                         const double *dlux, double ax, double al) {
  KQ_GATE(P);
  if (P.axal) { ax = P.axal[0]; al = P.axal[1]; }
  const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    S.x[i] += ax * z[i];
    if (P.haslx[i]) { S.slx[i] += ax * dslx[i]; S.llx[i] += al * dllx[i]; }
    if (P.hasux[i]) { S.sux[i] += ax * dsux[i]; S.lux[i] += al * dlux[i]; }
  }
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.m; a += (int64_t)gridDim.x * blockDim.x) {
    if (P.hasl[a]) { S.sl[a] += ax * dsl[a]; S.ll[a] += al * z[lo_off + a]; }
    if (P.hasu[a]) { S.su[a] += ax * dsu[a]; S.lu[a] += al * z[up_off + a]; }
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.me; e += (int64_t)gridDim.x * blockDim.x)
    S.le[e] += al * z[P.n + e];
}

__global__ void k_reduce_cols(int nb, int ncol, const double *part, int min_mask, double *out,
                              const int *gate) {
  if (gate && *gate == 0) return;
  __shared__ double sh[32];
  for (int c = 0; c < ncol; ++c) {
    if ((min_mask >> c) & 1) {
      double v = INFINITY;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) v = fmin(v, part[c * nb + i]);
      v = block_min(v, sh);
      if (threadIdx.x == 0) out[c] = v;
    } else {
      double s[1] = {0.0};
      for (int i = threadIdx.x; i < nb; i += blockDim.x) s[0] += part[c * nb + i];
      block_sum<1>(s, sh);
      if (threadIdx.x == 0) out[c] = s[0];
    }
    __syncthreads();
  }
}

// outputs in original units
__global__ void k_unscale(DevProb P, DevState S, double sigma, const double *rhoC, double *lA,
                          double *uA, double *lx, double *ux, double *le) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.m; a += (int64_t)gridDim.x * blockDim.x) {
    lA[a] = P.hasl[a] ? S.ll[a] * P.rhoA[a] / sigma : 0.0;
    uA[a] = P.hasu[a] ? S.lu[a] * P.rhoA[a] / sigma : 0.0;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    lx[i] = P.haslx[i] ? S.llx[i] / sigma : 0.0;
    ux[i] = P.hasux[i] ? S.lux[i] / sigma : 0.0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.me; e += (int64_t)gridDim.x * blockDim.x)
    le[e] = S.le[e] * rhoC[e] / sigma;
}

// adjoint gradients: grad_p = -sigma v,  grad_lA = -rho w_l,  grad_uA = rho w_u,  grad_b = -rhoC w_e
__global__ void k_adjoint_out(DevProb P, double sigma, const double *rhoC, const double *z, double *gp,
                              double *glA, double *guA, double *gb) {
  const int64_t lo_off = P.n + P.me, up_off = P.n + P.me + P.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x)
    gp[i] = -sigma * z[i];
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.m; a += (int64_t)gridDim.x * blockDim.x) {
    glA[a] = P.hasl[a] ? -P.rhoA[a] * z[lo_off + a] : 0.0;
    guA[a] = P.hasu[a] ? P.rhoA[a] * z[up_off + a] : 0.0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.me; e += (int64_t)gridDim.x * blockDim.x)
    gb[e] = -rhoC[e] * z[P.n + e];
}

__global__ void k_set_state_mask(DevProb P, DevState S) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!P.haslx[i]) { S.slx[i] = 1.0; S.llx[i] = 0.0; }
    if (!P.hasux[i]) { S.sux[i] = 1.0; S.lux[i] = 0.0; }
  }
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.m; a += (int64_t)gridDim.x * blockDim.x) {
    if (!P.hasl[a]) { S.sl[a] = 1.0; S.ll[a] = 0.0; }
    if (!P.hasu[a]) { S.su[a] = 1.0; S.lu[a] = 0.0; }
  }
}

__global__ void k_pad_rhs(int64_t N, const double *g, int64_t n, double *rhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    rhs[i] = i < n ? g[i] : 0.0;
}

// ---------------------------------------------------------------- host helpers
template <class X> X *dalloc(kq_problem *h, size_t count) {
  void *p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(X)) != cudaSuccess) return nullptr;
  cudaMemset(p, 0, std::max<size_t>(count, 1) * sizeof(X));
  h->allocs.push_back(p);
  return reinterpret_cast<X *>(p);
}

size_t dtype_size(int dt) { return dt == KQ_F64 ? 8 : (dt == KQ_F32 ? 4 : 2); }

kq_status rowdot(kq_problem *h, const double *v, double *t, double *tC) {
  const DevProb &P = h->P;
  if (P.m + P.me == 0) return KQ_OK;
  if (P.akind == KQ_A_CSR) {
    if (P.adtype == KQ_F32) k_rowdot_acsr<float><<<NB, NT, 0, h->stream>>>(P, v, t, tC);
    else k_rowdot_acsr<double><<<NB, NT, 0, h->stream>>>(P, v, t, tC);
  } else if (P.akind == KQ_A_ROWS_OF_P || (P.akind == KQ_A_NONE && P.hkind == KQ_H_CSR_LSQ))
    k_rowdot_prows<<<NB, NT, 0, h->stream>>>(P, v, t, tC);
  else if (P.adtype == KQ_F32)
    k_rowdot_dense<float><<<NB, NT, 0, h->stream>>>(P, v, t, tC);
  else
    k_rowdot_dense<double><<<NB, NT, 0, h->stream>>>(P, v, t, tC);
  ++h->launches;
  KQ_CUDA(h, cudaGetLastError());
  return KQ_OK;
}

kq_status hx_apply(kq_problem *h, const double *v, double *hx) {
  const DevProb &P = h->P;
  if (P.hkind == KQ_H_DENSE) {
    if (P.hdtype == KQ_F64) k_hx_dense<double><<<NB, NT, 0, h->stream>>>(P, v, hx);
    else if (P.hdtype == KQ_F32) k_hx_dense<float><<<NB, NT, 0, h->stream>>>(P, v, hx);
    else k_hx_dense<__nv_bfloat16><<<NB, NT, 0, h->stream>>>(P, v, hx);
    ++h->launches;
  } else if (P.hkind == KQ_H_LOWRANK) {
    KQ_CUDA(h, cudaMemsetAsync(h->g, 0, P.k * sizeof(double), h->stream));
    const int nbz = (int)std::min<int64_t>(1024, std::max<int64_t>(1, P.n / 64));
    if (P.hdtype == KQ_F64) {
      k_zt<double><<<nbz, 256, 0, h->stream>>>(P, v, h->g);
      ++h->launches;
      k_zg<double><<<NB, NT, 0, h->stream>>>(P, h->g, v, hx);
      ++h->launches;
    } else {
      k_zt<float><<<nbz, 256, 0, h->stream>>>(P, v, h->g);
      ++h->launches;
      k_zg<float><<<NB, NT, 0, h->stream>>>(P, h->g, v, hx);
      ++h->launches;
    }
  } else {
    // CSR: H x is produced by the scatter pass; here y = P x
    k_csr_rowdot<<<NB, NT, 0, h->stream>>>(P, v, h->yP);
    ++h->launches;
    KQ_CUDA(h, cudaMemsetAsync(hx, 0, P.n * sizeof(double), h->stream));
  }
  KQ_CUDA(h, cudaGetLastError());
  return KQ_OK;
}

}  // namespace

// Reduce ncols columns of block partials (sum, or min where bit c of min_mask
// is set) into h->h_red[off .. off+ncols) asynchronously (no host sync).
kq_status reduce_async(kq_problem *h, int ncols, int min_mask, int off) {
  k_reduce_cols<<<1, 256, 0, h->stream>>>(NB, ncols, h->red, min_mask, h->red_out + off,
                                           h->P.gate);
  ++h->launches;
  if (!h->graph_mode)   // in a captured graph the results stay on the device
    KQ_CUDA(h, cudaMemcpyAsync(h->h_red + off, h->red_out + off, ncols * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
  return KQ_OK;
}

namespace {

kq_status fetch(kq_problem *h, int ncols, std::vector<int> mins, double *out) {
  int mask = 0;
  for (size_t i = 0; i < mins.size(); ++i) mask |= (mins[i] ? 1 : 0) << i;
  kq_status rc = reduce_async(h, ncols, mask, 0);
  if (rc != KQ_OK) return rc;
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int c = 0; c < ncols; ++c) out[c] = h->h_red[c];
  return KQ_OK;
}

// initial point of the iteration (x0 from the bounds, slacks max(value, 1),
// inequality multipliers 1, lam_e 0)
}  // namespace

kq_status init_state(kq_problem *h) {
  k_init_x<<<NB, NT, 0, h->stream>>>(h->P, h->S);
  ++h->launches;
  if (h->m > 0) {
    kq_status rc = rowdot(h, h->S.x, h->t, h->tC);
    if (rc != KQ_OK) return rc;
  }
  k_init_rows<<<NB, NT, 0, h->stream>>>(h->P, h->S, h->t);
  ++h->launches;
  KQ_CUDA(h, cudaGetLastError());
  h->kkt_valid = false;
  return KQ_OK;
}

kq_status kq_fail(kq_problem *h, kq_status st, const std::string &msg) {
  if (h) h->err = msg;
  else g_global_err = msg;
  return st;
}

// Residuals, D, dg, doubly augmented rhs and Jacobi diagonal at (state, mu).
// Returns the squared residual norm pieces through h->h_red: [0] = |r|^2,
// [1] = |r_H|^2.
kq_status assemble_enqueue(kq_problem *h) {
  const DevProb &P = h->P;
  h->K.mu = h->mu;
  kq_status st;
  if ((st = hx_apply(h, h->S.x, h->hx)) != KQ_OK) return st;
  if ((st = rowdot(h, h->S.x, h->t, h->tC)) != KQ_OK) return st;
  RowCoef cf{h->acc1 + P.n, h->acc2 + P.n, h->acc3 + P.n};   // coefficient arrays share storage
  // zero the per-row and per-column accumulators
  KQ_CUDA(h, cudaMemsetAsync(h->acc1, 0, P.n * sizeof(double), h->stream));
  KQ_CUDA(h, cudaMemsetAsync(h->acc2, 0, P.n * sizeof(double), h->stream));
  KQ_CUDA(h, cudaMemsetAsync(h->acc3, 0, P.n * sizeof(double), h->stream));
  KQ_CUDA(h, cudaMemsetAsync(h->red, 0, 5 * NB * sizeof(double), h->stream));
  k_rows_resid<<<NB, NT, 0, h->stream>>>(P, h->S, h->K, h->t, h->tC, cf, h->red + 3 * NB);
  ++h->launches;
  if (P.hkind == KQ_H_CSR_LSQ) {
    // the rows of P (H x and, for ROWS_OF_P, the dose-limit rows)
    k_csr_scatter<<<NB * 4, NT, 0, h->stream>>>(P, h->yP, cf, h->acc1, h->acc2, h->acc3);
    ++h->launches;
  }
  if (P.akind == KQ_A_CSR && P.m > 0) {
    if (P.adtype == KQ_F32) k_acsr_scatter<float><<<NB * 4, NT, 0, h->stream>>>(P, cf, h->acc1, h->acc2, h->acc3);
    else k_acsr_scatter<double><<<NB * 4, NT, 0, h->stream>>>(P, cf, h->acc1, h->acc2, h->acc3);
    ++h->launches;
  }
  // dense general rows and the equality rows (k_rows_scatter_dense reads A
  // only when it is dense)
  if ((P.akind == KQ_A_DENSE && P.m > 0) || P.me > 0) {
    if (P.adtype == KQ_F32) k_rows_scatter_dense<float><<<NB, NT, 0, h->stream>>>(P, cf, h->acc1, h->acc2, h->acc3);
    else k_rows_scatter_dense<double><<<NB, NT, 0, h->stream>>>(P, cf, h->acc1, h->acc2, h->acc3);
    ++h->launches;
  }
  k_x_resid<<<NB, NT, 0, h->stream>>>(P, h->S, h->K, h->hx, h->acc1, h->acc2, h->acc3, h->red);
  ++h->launches;
  KQ_CUDA(h, cudaGetLastError());
  return reduce_async(h, 5, 0, 10);
}

// after a stream synchronisation: |r|^2 (all blocks of Eq. (7)) and |r_H|^2;
// the section 5.2 infeasibilities (squared) go to h->inf2 = [primal, dual, compl]
void assemble_finish(kq_problem *h, double *norm2, double *rH2) {
  const double *r = h->h_red + 10;   // [bound res, r_H, bound compl, row res, row compl]
  *norm2 = r[0] + r[1] + r[2] + r[3] + r[4];
  if (rH2) *rH2 = r[1];
  h->inf2[0] = r[0] + r[3];
  h->inf2[1] = r[1];
  h->inf2[2] = r[2] + r[4];
  h->kkt_valid = true;
}

static kq_status assemble_norms(kq_problem *h, double *norm2, double *rH2) {
  kq_status rc = assemble_enqueue(h);
  if (rc != KQ_OK) return rc;
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  assemble_finish(h, norm2, rH2);
  return KQ_OK;
}

// step recovery and ratio-test reductions for the direction in h->z
kq_status recover_enqueue(kq_problem *h) {
  kq_status rc = rowdot(h, h->z, h->t, h->tC);
  if (rc != KQ_OK) return rc;
  k_recover_ratio<<<NB, NT, 0, h->stream>>>(h->P, h->S, h->K, h->z, h->t, h->dsl, h->dsu, h->dslx,
                                             h->dsux, h->dllx, h->dlux, h->red);
  ++h->launches;
  return reduce_async(h, 2, 3, 4);
}

void recover_finish(kq_problem *h, double gamma, double *ax, double *al) {
  *ax = std::min(1.0, gamma * h->h_red[4]);
  *al = std::min(1.0, gamma * h->h_red[5]);
}

kq_status update_enqueue(kq_problem *h, double ax, double al) {
  k_update<<<NB, NT, 0, h->stream>>>(h->P, h->S, h->z, h->dsl, h->dsu, h->dslx, h->dsux, h->dllx,
                                      h->dlux, ax, al);
  ++h->launches;
  KQ_CUDA(h, cudaGetLastError());
  return KQ_OK;
}

// x and the multipliers in original units into caller buffers (async)
kq_status outputs_enqueue(kq_problem *h, double *x, double *lam_lA, double *lam_uA,
                          double *lam_lx, double *lam_ux, double *lam_e) {
  const size_t nb = h->n * 8;
  if (x) KQ_CUDA(h, cudaMemcpyAsync(x, h->S.x, nb, cudaMemcpyDefault, h->stream));
  if (lam_lA || lam_uA || lam_lx || lam_ux || lam_e) {
    double *olA = h->tmp + h->n + h->me, *ouA = h->tmp + h->n + h->me + h->m, *olx = h->acc2,
           *oux = h->acc3, *oe = h->tmp + h->n;
    k_unscale<<<NB, NT, 0, h->stream>>>(h->P, h->S, h->sigma, h->rhoC, olA, ouA, olx, oux, oe);
    ++h->launches;
    if (lam_lA && h->m) KQ_CUDA(h, cudaMemcpyAsync(lam_lA, olA, h->m * 8, cudaMemcpyDefault, h->stream));
    if (lam_uA && h->m) KQ_CUDA(h, cudaMemcpyAsync(lam_uA, ouA, h->m * 8, cudaMemcpyDefault, h->stream));
    if (lam_lx) KQ_CUDA(h, cudaMemcpyAsync(lam_lx, olx, nb, cudaMemcpyDefault, h->stream));
    if (lam_ux) KQ_CUDA(h, cudaMemcpyAsync(lam_ux, oux, nb, cudaMemcpyDefault, h->stream));
    if (lam_e && h->me) KQ_CUDA(h, cudaMemcpyAsync(lam_e, oe, h->me * 8, cudaMemcpyDefault, h->stream));
    h->kkt_valid = false;
  }
  return KQ_OK;
}

// small vector helpers used by the batched solver
__global__ void k_vec_add(int64_t N, double *z, const double *dz, const int *gate) {
  if (gate && *gate == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += dz[i];
}
__global__ void k_vec_resid(int64_t N, const double *rhs, const double *kz, double *res, double *part,
                            const int *gate) {
  if (gate && *gate == 0) return;
  __shared__ double sh[32];
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = rhs[i] - kz[i];
    res[i] = v;
    s[0] += v * v;
  }
  block_sum<1>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}
kq_status vec_add_enqueue(kq_problem *h, double *z, const double *dz) {
  const int nb = (int)std::min<int64_t>(NB, ceil_div64(h->nkp, NT));
  k_vec_add<<<nb, NT, 0, h->stream>>>(h->nkp, z, dz, h->vec_gate);
  ++h->launches;
  return KQ_OK;
}
// res = rhs - kz and |res|^2 into h->h_red[8] (async)
kq_status vec_resid_enqueue(kq_problem *h, const double *rhs, const double *kz, double *res) {
  KQ_CUDA(h, cudaMemsetAsync(h->red, 0, NB * sizeof(double), h->stream));
  const int nb = (int)std::min<int64_t>(NB, ceil_div64(h->nkp, NT));
  k_vec_resid<<<nb, NT, 0, h->stream>>>(h->nkp, rhs, kz, res, h->red, h->vec_gate);
  ++h->launches;
  return reduce_async(h, 1, 0, 8);
}


kq_status kkt_assemble(kq_problem *h) {
  double n2;
  return assemble_norms(h, &n2, nullptr);
}

// ---------------------------------------------------------------- C ABI
extern "C" {

void kq_default_ipm_opts(kq_ipm_opts *o) {
  if (!o) return;
  o->gamma = 0.99;
  o->mu0 = 1.0;
  o->mu_tol = 1e-6;
  o->ipm_maxit = 200;
  o->pcg_tol = 1e-7;
  o->pcg_maxit = 5000;
  o->precision = KQ_PREC_F64;
  o->refine_steps = 6;
  o->inner_tol = 1e-4;
  o->timeout_s = 2.0;
  o->grid_ctas = 0;
  o->verbose = 0;
  o->record = 0;
  o->graph = 1;
  o->warm_start = 0;
}

void kq_default_pcg_opts(kq_pcg_opts *o) {
  if (!o) return;
  o->tol = 1e-7;
  o->maxit = 5000;
  o->precision = KQ_PREC_F64;
  o->refine_steps = 6;
  o->inner_tol = 1e-4;
}

const char *kq_global_error(void) { return g_global_err.c_str(); }
const char *qp_last_error(kq_handle h) { return h ? h->err.c_str() : g_global_err.c_str(); }

void qp_destroy(kq_handle h) {
  if (!h) return;
  for (void *p : h->allocs) cudaFree(p);
  if (h->h_red) cudaFreeHost(h->h_red);
  if (h->W.h_pinned) cudaFreeHost(h->W.h_pinned);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

kq_status qp_create(kq_handle *out, int64_t n, const kq_hop *H, const double *p,
                    const kq_amat *A, const double *lA, const double *uA, int64_t me,
                    const double *C, const double *b, const double *lx, const double *ux,
                    void *stream) {
  if (!out) return kq_fail(nullptr, KQ_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !H || !p) return kq_fail(nullptr, KQ_ERR_ARG, "n <= 0, H or p missing");
  const int akind = A ? A->kind : KQ_A_NONE;
  const int64_t m = (akind == KQ_A_NONE) ? 0 : A->m;
  if (m < 0 || me < 0) return kq_fail(nullptr, KQ_ERR_ARG, "negative row count");
  if (m > 0 && (!lA || !uA)) return kq_fail(nullptr, KQ_ERR_ARG, "lA/uA required when A has rows");
  if (me > 0 && (!C || !b)) return kq_fail(nullptr, KQ_ERR_ARG, "C/b required when me > 0");
  if (H->kind == KQ_H_CSR_LSQ) {
    if (akind == KQ_A_DENSE)
      return kq_fail(nullptr, KQ_ERR_ARG, "CSR_LSQ H supports A = NONE, CSR or ROWS_OF_P");
    if (H->dtype != KQ_F32 || H->cols != n || !H->val || !H->col || !H->rowptr || !H->w)
      return kq_fail(nullptr, KQ_ERR_ARG, "CSR_LSQ needs F32 values, col, rowptr, w and cols == n");
  } else if (H->kind == KQ_H_DENSE) {
    if (akind == KQ_A_ROWS_OF_P) return kq_fail(nullptr, KQ_ERR_ARG, "ROWS_OF_P needs CSR_LSQ H");
    if (!H->val) return kq_fail(nullptr, KQ_ERR_ARG, "dense H values missing");
  } else if (H->kind == KQ_H_RBF) {
    if (akind == KQ_A_ROWS_OF_P) return kq_fail(nullptr, KQ_ERR_ARG, "ROWS_OF_P needs CSR_LSQ H");
    if (!H->val || H->rows != n || H->cols <= 0 || !(H->gamma > 0.0) || isinf(H->gamma) ||
        n > (int64_t)65535 * 32 ||
        (H->dtype != KQ_F64 && H->dtype != KQ_F32 && H->dtype != KQ_BF16))
      return kq_fail(nullptr, KQ_ERR_ARG, "RBF needs X (n x d, d > 0), finite gamma > 0 and an H storage type");
  } else if (H->kind == KQ_H_LOWRANK) {
    if (akind != KQ_A_NONE && akind != KQ_A_CSR)
      return kq_fail(nullptr, KQ_ERR_ARG, "LOWRANK H supports A = NONE or CSR");
    if (!H->val || H->rows != n || H->cols <= 0 || H->dtype == KQ_BF16)
      return kq_fail(nullptr, KQ_ERR_ARG, "LOWRANK needs Z (n x k, F32/F64)");
  } else {
    return kq_fail(nullptr, KQ_ERR_ARG, "unknown H kind");
  }
  if (akind == KQ_A_DENSE && (!A->val || (A->dtype != KQ_F64 && A->dtype != KQ_F32)))
    return kq_fail(nullptr, KQ_ERR_ARG, "dense A needs F64 or F32 values");
  if (akind == KQ_A_ROWS_OF_P && !A->rows) return kq_fail(nullptr, KQ_ERR_ARG, "ROWS_OF_P needs rows");
  if (akind == KQ_A_CSR && (A->nnz < 0 || (A->nnz > 0 && (!A->val || !A->col)) || !A->rowptr ||
                            (A->dtype != KQ_F64 && A->dtype != KQ_F32)))
    return kq_fail(nullptr, KQ_ERR_ARG, "CSR A needs F64 or F32 values, col, rowptr and nnz >= 0");
  if (akind != KQ_A_NONE && akind != KQ_A_DENSE && akind != KQ_A_CSR && akind != KQ_A_ROWS_OF_P)
    return kq_fail(nullptr, KQ_ERR_ARG, "unknown A kind");

  kq_problem *h = new kq_problem();
  h->stream = (cudaStream_t)stream;
  h->n = n; h->m = m; h->me = me; h->nkp = n + me + 2 * m;
  DevProb &P = h->P;
  P.n = n; P.m = m; P.me = me; P.nkp = h->nkp;
  // an RBF-kernel H is formed once and then used as a stored dense H
  P.hkind = H->kind == KQ_H_RBF ? KQ_H_DENSE : H->kind;
  P.hdtype = H->dtype; P.akind = akind;
  P.adtype = (akind == KQ_A_DENSE || akind == KQ_A_CSR) ? A->dtype : KQ_F64;
  auto fail = [&](kq_status st, const std::string &msg) {
    g_global_err = msg;
    qp_destroy(h);
    return st;
  };
  if (cudaGetDevice(&h->dev) != cudaSuccess) return fail(KQ_ERR_CUDA, "no CUDA device");
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev);
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess)
    return fail(KQ_ERR_CUDA, "event create");
  if (cudaMallocHost((void **)&h->h_red, 64 * sizeof(double)) != cudaSuccess) return fail(KQ_ERR_OOM, "pinned");
  cudaStream_t s = h->stream;
  auto up = [&](const void *src, size_t bytes) -> void * {
    void *d = nullptr;
    if (cudaMalloc(&d, std::max<size_t>(bytes, 8)) != cudaSuccess) return nullptr;
    h->allocs.push_back(d);
    if (src && bytes) cudaMemcpyAsync(d, src, bytes, cudaMemcpyDefault, s);
    else cudaMemsetAsync(d, 0, std::max<size_t>(bytes, 8), s);
    return d;
  };
  // ---- H
  double *hdiag = dalloc<double>(h, n);
  if (!hdiag) return fail(KQ_ERR_OOM, "hdiag");
  if (H->kind == KQ_H_DENSE) {
    // rows padded with zeros to a multiple of 8 entries (16-byte aligned rows)
    P.hld = (n + 7) & ~(int64_t)7;
    const size_t es = dtype_size(H->dtype);
    P.Hd = up(nullptr, (size_t)n * P.hld * es);
    if (!P.Hd) return fail(KQ_ERR_OOM, "H");
    if (cudaMemcpy2DAsync((void *)P.Hd, P.hld * es, H->val, n * es, n * es, n, cudaMemcpyDefault, s) != cudaSuccess)
      return fail(KQ_ERR_CUDA, "H upload");
    if (H->dtype == KQ_F64)
      k_dense_diag<double><<<NB, NT, 0, s>>>(n, P.hld, (const double *)P.Hd, hdiag);
    else if (H->dtype == KQ_F32)
      k_dense_diag<float><<<NB, NT, 0, s>>>(n, P.hld, (const float *)P.Hd, hdiag);
    else
      k_dense_diag<__nv_bfloat16><<<NB, NT, 0, s>>>(n, P.hld, (const __nv_bfloat16 *)P.Hd, hdiag);
  } else if (H->kind == KQ_H_RBF) {
    // samples and labels are needed only while H is formed
    P.hld = (n + 7) & ~(int64_t)7;
    const size_t es = dtype_size(H->dtype);
    P.Hd = up(nullptr, (size_t)n * P.hld * es);
    if (!P.Hd) return fail(KQ_ERR_OOM, "H");
    const int64_t d = H->cols;
    double *Xd = nullptr, *yd = nullptr;
    if (cudaMalloc((void **)&Xd, (size_t)n * d * sizeof(double)) != cudaSuccess)
      return fail(KQ_ERR_OOM, "RBF samples");
    if (H->w && cudaMalloc((void **)&yd, (size_t)n * sizeof(double)) != cudaSuccess) {
      cudaFree(Xd);
      return fail(KQ_ERR_OOM, "RBF labels");
    }
    cudaError_t e = cudaMemcpyAsync(Xd, H->val, (size_t)n * d * sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess && yd) e = cudaMemcpyAsync(yd, H->w, (size_t)n * sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess) {
      const dim3 grid((unsigned)ceil_div64(n, 32), (unsigned)ceil_div64(n, 32));
      if (H->dtype == KQ_F64)
        k_rbf_build<double><<<grid, 256, 0, s>>>(n, d, Xd, yd, H->gamma, P.hld, (double *)P.Hd);
      else if (H->dtype == KQ_F32)
        k_rbf_build<float><<<grid, 256, 0, s>>>(n, d, Xd, yd, H->gamma, P.hld, (float *)P.Hd);
      else
        k_rbf_build<__nv_bfloat16><<<grid, 256, 0, s>>>(n, d, Xd, yd, H->gamma, P.hld,
                                                        (__nv_bfloat16 *)P.Hd);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(Xd);
    if (yd) cudaFree(yd);
    if (e != cudaSuccess) return fail(KQ_ERR_CUDA, std::string("RBF build: ") + cudaGetErrorString(e));
    if (H->dtype == KQ_F64) k_dense_diag<double><<<NB, NT, 0, s>>>(n, P.hld, (const double *)P.Hd, hdiag);
    else if (H->dtype == KQ_F32) k_dense_diag<float><<<NB, NT, 0, s>>>(n, P.hld, (const float *)P.Hd, hdiag);
    else k_dense_diag<__nv_bfloat16><<<NB, NT, 0, s>>>(n, P.hld, (const __nv_bfloat16 *)P.Hd, hdiag);
  } else if (H->kind == KQ_H_LOWRANK) {
    P.k = H->cols;
    P.Z = up(H->val, (size_t)n * P.k * dtype_size(H->dtype));
    if (!P.Z) return fail(KQ_ERR_OOM, "Z");
    if (H->w) {
      P.zw = (const double *)up(H->w, P.k * sizeof(double));
      if (!P.zw) return fail(KQ_ERR_OOM, "Z weights");
    }
    if (H->d0) {
      P.d0 = (const double *)up(H->d0, n * sizeof(double));
      if (!P.d0) return fail(KQ_ERR_OOM, "H0");
    }
    if (H->dtype == KQ_F64) k_rownorm2<double><<<NB, NT, 0, s>>>(n, P.k, (const double *)P.Z, P.zw, P.d0, hdiag);
    else k_rownorm2<float><<<NB, NT, 0, s>>>(n, P.k, (const float *)P.Z, P.zw, P.d0, hdiag);
  } else {
    P.nP = H->rows;
    int64_t nnz = H->nnz;
    P.rowptr = (const int64_t *)up(H->rowptr, (P.nP + 1) * sizeof(int64_t));
    // pad value/col arrays by 128 elements so that vector tails stay in bounds
    P.col = (const int32_t *)up(nullptr, (nnz + 128) * sizeof(int32_t));
    P.val = (const float *)up(nullptr, (nnz + 128) * sizeof(float));
    double *w2 = (double *)up(H->w, P.nP * sizeof(double));
    P.w2 = w2;
    int32_t *p2a = (int32_t *)up(nullptr, P.nP * sizeof(int32_t));
    P.prow2a = p2a;
    if (!P.rowptr || !P.col || !P.val || !w2 || !p2a) return fail(KQ_ERR_OOM, "P");
    cudaMemcpyAsync((void *)P.col, H->col, nnz * sizeof(int32_t), cudaMemcpyDefault, s);
    cudaMemcpyAsync((void *)P.val, H->val, nnz * sizeof(float), cudaMemcpyDefault, s);
    cudaMemsetAsync(p2a, 0xff, P.nP * sizeof(int32_t), s);
    P.nnz = nnz;
    {
      int *bad = dalloc<int>(h, 1);
      int32_t *rows_chk = nullptr;
      const int64_t mchk = (akind == KQ_A_ROWS_OF_P) ? m : 0;
      if (mchk) {
        rows_chk = (int32_t *)up(A->rows, m * sizeof(int32_t));
        if (!rows_chk) return fail(KQ_ERR_OOM, "rows");
      }
      if (!bad) return fail(KQ_ERR_OOM, "check flag");
      k_check_csr<<<NB, NT, 0, s>>>(P.nP, n, nnz, P.rowptr, P.col, mchk, rows_chk, bad);
      int hbad = 0;
      cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return fail(KQ_ERR_CUDA, "csr check");
      if (hbad) return fail(KQ_ERR_ARG, "invalid CSR structure (rowptr, col or rows out of range)");
      P.arows = rows_chk;
    }
    k_csr_diag<<<NB * 4, NT, 0, s>>>(P.nP, P.rowptr, P.col, P.val, w2, 2.0, hdiag);
  }
  // ---- sigma = 1 / max(1, max_i H_ii, |p|_inf)
  double *pd = (double *)up(p, n * sizeof(double));
  double *red = dalloc<double>(h, 8 * NB);
  double *red_out = dalloc<double>(h, 64);
  if (!pd || !red || !red_out) return fail(KQ_ERR_OOM, "p");
  h->red = red; h->red_out = red_out;
  k_max_abs<<<NB, NT, 0, s>>>(n, hdiag, red);
  k_max_abs<<<NB, NT, 0, s>>>(n, pd, red + NB);
  h->dflags = dalloc<int>(h, 8);
  if (!h->dflags) return fail(KQ_ERR_OOM, "flags");
  {
    // max of the block partials as the min of their negatives
    k_scale_vec<<<NB, NT, 0, s>>>(2 * NB, red, nullptr, -1.0);
    if (fetch(h, 2, {1, 1}, h->h_red + 40) != KQ_OK) return fail(KQ_ERR_CUDA, "create reduction");
    h->h_red[0] = h->h_red[40];
    h->h_red[1] = h->h_red[41];
  }
  const double hmax = -h->h_red[0], pmax = -h->h_red[1];
  if (!(hmax == hmax) || !(pmax == pmax) || isinf(hmax) || isinf(pmax))
    return fail(KQ_ERR_NUMERIC, "H or p has NaN/Inf");
  const double sigma = 1.0 / std::max(1.0, std::max(hmax, pmax));
  h->sigma = sigma;
  h->sigma_create = sigma;
  h->hmax = hmax;
  k_scale_vec<<<NB, NT, 0, s>>>(n, pd, nullptr, sigma);
  k_scale_vec<<<NB, NT, 0, s>>>(n, hdiag, nullptr, sigma);
  P.p = pd;
  P.hscale = sigma;
  if (H->kind == KQ_H_CSR_LSQ) {
    k_scale_vec<<<NB, NT, 0, s>>>(P.nP, (double *)P.w2, nullptr, 2.0 * sigma);
    cudaMemsetAsync(hdiag, 0, n * sizeof(double), s);   // the pass adds diag(H)
  }
  P.hdiag = hdiag;
  // ---- general rows
  double *rhoA = dalloc<double>(h, m), *lAd = (double *)up(lA, m * sizeof(double)),
         *uAd = (double *)up(uA, m * sizeof(double));
  uint8_t *hl = dalloc<uint8_t>(h, m), *hu = dalloc<uint8_t>(h, m);
  if (!rhoA || !lAd || !uAd || !hl || !hu) return fail(KQ_ERR_OOM, "A");
  if (akind == KQ_A_DENSE) {
    P.ald = (n + 7) & ~(int64_t)7;
    const size_t es = dtype_size(A->dtype);
    P.Ad = up(nullptr, (size_t)m * P.ald * es);
    if (!P.Ad) return fail(KQ_ERR_OOM, "A values");
    if (m > 0 && cudaMemcpy2DAsync((void *)P.Ad, P.ald * es, A->val, n * es, n * es, m, cudaMemcpyDefault, s) != cudaSuccess)
      return fail(KQ_ERR_CUDA, "A upload");
    if (A->dtype == KQ_F64) k_rho_dense<double><<<NB, NT, 0, s>>>(m, n, P.ald, (const double *)P.Ad, rhoA);
    else k_rho_dense<float><<<NB, NT, 0, s>>>(m, n, P.ald, (const float *)P.Ad, rhoA);
  } else if (akind == KQ_A_CSR) {
    const size_t es = dtype_size(A->dtype);
    const int64_t annz = A->nnz;
    P.arowptr = (const int64_t *)up(A->rowptr, (m + 1) * sizeof(int64_t));
    P.acol = (const int32_t *)up(A->col, std::max<int64_t>(annz, 1) * sizeof(int32_t));
    P.aval = up(A->val, std::max<int64_t>(annz, 1) * es);
    P.annz = annz;
    int *bad = dalloc<int>(h, 1);
    if (!P.arowptr || !P.acol || !P.aval || !bad) return fail(KQ_ERR_OOM, "CSR A");
    if (annz == 0) {
      cudaMemsetAsync((void *)P.acol, 0, sizeof(int32_t), s);
      cudaMemsetAsync((void *)P.aval, 0, es, s);
    }
    k_check_csr<<<NB, NT, 0, s>>>(m, n, annz, P.arowptr, P.acol, 0, nullptr, bad);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(KQ_ERR_CUDA, "CSR A check");
    if (hbad) return fail(KQ_ERR_ARG, "invalid CSR structure of A (rowptr or col out of range)");
    if (A->dtype == KQ_F64) k_rho_acsr<double><<<NB, NT, 0, s>>>(m, P.arowptr, (const double *)P.aval, rhoA);
    else k_rho_acsr<float><<<NB, NT, 0, s>>>(m, P.arowptr, (const float *)P.aval, rhoA);
  } else if (akind == KQ_A_ROWS_OF_P) {
    const int32_t *rows = P.arows;   // uploaded and checked with the CSR structure
    k_rho_rows<<<NB, NT, 0, s>>>(m, rows, P.rowptr, P.val, rhoA);
    k_prow2a<<<NB, NT, 0, s>>>(m, rows, (int32_t *)P.prow2a);
  }
  if (m > 0) {
    k_flags<<<NB, NT, 0, s>>>(m, lAd, uAd, hl, hu);
    k_scale_vec<<<NB, NT, 0, s>>>(m, lAd, rhoA, 0.0);
    k_scale_vec<<<NB, NT, 0, s>>>(m, uAd, rhoA, 0.0);
  }
  P.rhoA = rhoA; P.lA = lAd; P.uA = uAd; P.hasl = hl; P.hasu = hu;
  // ---- equality rows
  double *Cd = (double *)up(C, (size_t)me * n * sizeof(double));
  double *bd = (double *)up(b, me * sizeof(double));
  double *rhoC = dalloc<double>(h, me);
  if (!Cd || !bd || !rhoC) return fail(KQ_ERR_OOM, "C");
  if (me > 0) k_scale_rows<<<(unsigned)me, 256, 0, s>>>(me, n, Cd, bd, rhoC);
  P.Cd = Cd; P.b = bd;
  h->rhoC = rhoC;
  h->g = dalloc<double>(h, std::max<int64_t>(P.k, 1) + me + 1);
  // ---- variable bounds
  std::vector<double> inf_lo, inf_hi;
  const double *lxs = lx, *uxs = ux;
  if (!lx) { inf_lo.assign(n, -INFINITY); lxs = inf_lo.data(); }
  if (!ux) { inf_hi.assign(n, INFINITY); uxs = inf_hi.data(); }
  double *lxd = (double *)up(lxs, n * sizeof(double)), *uxd = (double *)up(uxs, n * sizeof(double));
  uint8_t *hlx = dalloc<uint8_t>(h, n), *hux = dalloc<uint8_t>(h, n);
  if (!lxd || !uxd || !hlx || !hux) return fail(KQ_ERR_OOM, "bounds");
  k_flags<<<NB, NT, 0, s>>>(n, lxd, uxd, hlx, hux);
  P.lx = lxd; P.ux = uxd; P.haslx = hlx; P.hasux = hux;
  // ---- state, KKT data, scratch
  DevState &S = h->S;
  S.x = dalloc<double>(h, n); S.slx = dalloc<double>(h, n); S.sux = dalloc<double>(h, n);
  S.llx = dalloc<double>(h, n); S.lux = dalloc<double>(h, n);
  S.sl = dalloc<double>(h, m); S.su = dalloc<double>(h, m); S.ll = dalloc<double>(h, m);
  S.lu = dalloc<double>(h, m); S.le = dalloc<double>(h, me);
  DevKKT &K = h->K;
  K.Dl = dalloc<double>(h, m); K.Du = dalloc<double>(h, m); K.cl = dalloc<double>(h, m);
  K.cu = dalloc<double>(h, m); K.dg = dalloc<double>(h, n);
  K.diag = dalloc<double>(h, h->nkp); K.rhs = dalloc<double>(h, h->nkp);
  K.rH = dalloc<double>(h, n); K.rlx = dalloc<double>(h, n); K.rux = dalloc<double>(h, n);
  K.rc3 = dalloc<double>(h, n); K.rc4 = dalloc<double>(h, n);
  K.rlA = dalloc<double>(h, m); K.ruA = dalloc<double>(h, m); K.rc1 = dalloc<double>(h, m);
  K.rc2 = dalloc<double>(h, m); K.re = dalloc<double>(h, me);
  h->hx = dalloc<double>(h, n); h->t = dalloc<double>(h, m); h->tC = dalloc<double>(h, me);
  h->acc1 = dalloc<double>(h, n + m + me); h->acc2 = dalloc<double>(h, n + m + me);
  h->acc3 = dalloc<double>(h, n + m + me);
  h->yP = dalloc<double>(h, P.hkind == KQ_H_CSR_LSQ ? P.nP : 1);
  h->z = dalloc<double>(h, h->nkp); h->zref = dalloc<double>(h, h->nkp); h->tmp = dalloc<double>(h, h->nkp);
  h->dsl = dalloc<double>(h, m); h->dsu = dalloc<double>(h, m); h->dslx = dalloc<double>(h, n);
  h->dsux = dalloc<double>(h, n); h->dllx = dalloc<double>(h, n); h->dlux = dalloc<double>(h, n);
  if (!S.x || !S.le || !K.diag || !K.rhs || !h->acc3 || !h->yP || !h->z || !h->tmp || !h->dlux)
    return fail(KQ_ERR_OOM, "state/work");
  if (init_state(h) != KQ_OK) return fail(KQ_ERR_CUDA, h->err);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail(KQ_ERR_CUDA, "create kernels failed");
  kq_status rc = pcg_setup(h, 0);
  if (rc != KQ_OK) return fail(rc, h->err);
  h->mu = 1.0;
  h->mu_exp = 0;
  *out = h;
  return KQ_OK;
}

kq_status qp_update(kq_handle h, const double *p, const double *lA, const double *uA,
                    const double *b) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  DevProb &P = h->P;
  cudaStream_t s = h->stream;
  const int64_t n = h->n, m = h->m, me = h->me;
  if (p) {
    double *pd = const_cast<double *>(P.p);
    KQ_CUDA(h, cudaMemcpyAsync(pd, p, n * sizeof(double), cudaMemcpyDefault, s));
    k_max_abs<<<NB, NT, 0, s>>>(n, pd, h->red);
    k_scale_vec<<<NB, NT, 0, s>>>(NB, h->red, nullptr, -1.0);
    double pm[1];
    if (fetch(h, 1, {1}, pm) != KQ_OK) return kq_fail(h, KQ_ERR_CUDA, "qp_update: reduction");
    const double pmax = -pm[0];
    if (!(pmax == pmax) || isinf(pmax)) return kq_fail(h, KQ_ERR_NUMERIC, "qp_update: p has NaN/Inf");
    // the same objective scale rule as qp_create
    const double sigma = 1.0 / std::max(1.0, std::max(h->hmax, pmax));
    const double ratio = sigma / h->sigma;
    k_scale_vec<<<NB, NT, 0, s>>>(n, pd, nullptr, sigma);
    if (ratio != 1.0) {
      if (P.hkind == KQ_H_CSR_LSQ) {
        k_scale_vec<<<NB, NT, 0, s>>>(P.nP, const_cast<double *>(P.w2), nullptr, ratio);
        P.wfac = sigma / h->sigma_create;
        P.wfac32 = (float)P.wfac;
      } else {
        k_scale_vec<<<NB, NT, 0, s>>>(n, const_cast<double *>(P.hdiag), nullptr, ratio);
        P.hscale = sigma;
      }
      h->sigma = sigma;
    }
  }
  if (m > 0 && (lA || uA)) {
    double *lAd = const_cast<double *>(P.lA), *uAd = const_cast<double *>(P.uA);
    if (lA) KQ_CUDA(h, cudaMemcpyAsync(lAd, lA, m * sizeof(double), cudaMemcpyDefault, s));
    if (uA) KQ_CUDA(h, cudaMemcpyAsync(uAd, uA, m * sizeof(double), cudaMemcpyDefault, s));
    // the row scaling of qp_create applied to the replaced bounds (the others
    // are stored scaled already), then the flags from finiteness
    k_flags_scaled<<<NB, NT, 0, s>>>(m, lAd, uAd, lA != nullptr, uA != nullptr, P.rhoA,
                                      const_cast<uint8_t *>(P.hasl), const_cast<uint8_t *>(P.hasu));
  }
  if (me > 0 && b) {
    double *bd = const_cast<double *>(P.b);
    KQ_CUDA(h, cudaMemcpyAsync(bd, b, me * sizeof(double), cudaMemcpyDefault, s));
    k_scale_vec<<<NB, NT, 0, s>>>(me, bd, h->rhoC, 0.0);
  }
  KQ_CUDA(h, cudaGetLastError());
  KQ_CUDA(h, cudaStreamSynchronize(s));
  h->solved = false;
  h->state_set = false;
  h->kkt_valid = false;
  return KQ_OK;
}

kq_status qp_iteration_log(kq_handle h, kq_ipm_iter *out, int cap, int *count) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  if (!h->record && h->iter_log.empty())
    return kq_fail(h, KQ_ERR_STATE, "no ipm_solve with opts.record = 1 ran");
  const int k = (int)h->iter_log.size();
  if (count) *count = k;
  if (out)
    for (int i = 0; i < std::min(k, std::max(cap, 0)); ++i) out[i] = h->iter_log[i];
  return KQ_OK;
}

kq_status qp_sizes(kq_handle h, int64_t *n, int64_t *m, int64_t *me, int64_t *nkp) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  if (n) *n = h->n;
  if (m) *m = h->m;
  if (me) *me = h->me;
  if (nkp) *nkp = h->nkp;
  return KQ_OK;
}

kq_status qp_scaling(kq_handle h, double *sigma, double *rhoA, double *rhoC) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  if (sigma) *sigma = h->sigma;
  if (rhoA && h->m) KQ_CUDA(h, cudaMemcpyAsync(rhoA, h->P.rhoA, h->m * 8, cudaMemcpyDefault, h->stream));
  if (rhoC && h->me)
    KQ_CUDA(h, cudaMemcpyAsync(rhoC, h->rhoC, h->me * 8, cudaMemcpyDefault, h->stream));
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  return KQ_OK;
}

kq_status qp_get_state(kq_handle h, double *x, double *s_lA, double *s_uA, double *s_lx,
                       double *s_ux, double *lam_lA, double *lam_uA, double *lam_lx,
                       double *lam_ux, double *lam_e, double *mu) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  const size_t nb = h->n * 8, mb = h->m * 8, eb = h->me * 8;
  struct { double *dst; const double *src; size_t b; } c[] = {
      {x, h->S.x, nb}, {s_lA, h->S.sl, mb}, {s_uA, h->S.su, mb}, {s_lx, h->S.slx, nb},
      {s_ux, h->S.sux, nb}, {lam_lA, h->S.ll, mb}, {lam_uA, h->S.lu, mb}, {lam_lx, h->S.llx, nb},
      {lam_ux, h->S.lux, nb}, {lam_e, h->S.le, eb}};
  for (auto &e : c)
    if (e.dst && e.b) KQ_CUDA(h, cudaMemcpyAsync(e.dst, e.src, e.b, cudaMemcpyDefault, h->stream));
  if (mu) *mu = h->mu;
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  return KQ_OK;
}

kq_status qp_set_state(kq_handle h, const double *x, const double *s_lA, const double *s_uA,
                       const double *s_lx, const double *s_ux, const double *lam_lA,
                       const double *lam_uA, const double *lam_lx, const double *lam_ux,
                       const double *lam_e, double mu) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  if (!(mu > 0.0)) return kq_fail(h, KQ_ERR_ARG, "mu must be positive");
  const size_t nb = h->n * 8, mb = h->m * 8, eb = h->me * 8;
  struct { double *dst; const double *src; size_t b; } c[] = {
      {h->S.x, x, nb}, {h->S.sl, s_lA, mb}, {h->S.su, s_uA, mb}, {h->S.slx, s_lx, nb},
      {h->S.sux, s_ux, nb}, {h->S.ll, lam_lA, mb}, {h->S.lu, lam_uA, mb}, {h->S.llx, lam_lx, nb},
      {h->S.lux, lam_ux, nb}, {h->S.le, lam_e, eb}};
  for (auto &e : c)
    if (e.src && e.b) KQ_CUDA(h, cudaMemcpyAsync(e.dst, e.src, e.b, cudaMemcpyDefault, h->stream));
  k_set_state_mask<<<NB, NT, 0, h->stream>>>(h->P, h->S);
  ++h->launches;
  KQ_CUDA(h, cudaGetLastError());
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  h->mu = mu;
  h->mu_exp = 0;
  h->kkt_valid = false;
  h->state_set = true;
  return KQ_OK;
}

kq_status qp_residuals(kq_handle h, double *r_H, double *r_lA, double *r_uA, double *r_c1,
                       double *r_c2, double *r_lx, double *r_ux, double *r_c3, double *r_c4,
                       double *r_e, double *rhs, double *norm) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  double n2;
  kq_status rc = assemble_norms(h, &n2, nullptr);
  if (rc != KQ_OK) return rc;
  const size_t nb = h->n * 8, mb = h->m * 8, eb = h->me * 8;
  struct { double *dst; const double *src; size_t b; } c[] = {
      {r_H, h->K.rH, nb}, {r_lA, h->K.rlA, mb}, {r_uA, h->K.ruA, mb}, {r_c1, h->K.rc1, mb},
      {r_c2, h->K.rc2, mb}, {r_lx, h->K.rlx, nb}, {r_ux, h->K.rux, nb}, {r_c3, h->K.rc3, nb},
      {r_c4, h->K.rc4, nb}, {r_e, h->K.re, eb}, {rhs, h->K.rhs, (size_t)h->nkp * 8}};
  for (auto &e : c)
    if (e.dst && e.b) KQ_CUDA(h, cudaMemcpyAsync(e.dst, e.src, e.b, cudaMemcpyDefault, h->stream));
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  if (norm) *norm = sqrt(n2);
  return KQ_OK;
}

kq_status kkt_diag(kq_handle h, double *diag) {
  if (!h || !diag) return kq_fail(h, KQ_ERR_ARG, "null argument");
  if (!h->kkt_valid) { kq_status rc = kkt_assemble(h); if (rc != KQ_OK) return rc; }
  KQ_CUDA(h, cudaMemcpyAsync(diag, h->K.diag, h->nkp * 8, cudaMemcpyDefault, h->stream));
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  return KQ_OK;
}

kq_status kkt_apply(kq_handle h, const double *v, double *out, int precision) {
  if (!h || !v || !out) return kq_fail(h, KQ_ERR_ARG, "null argument");
  if (!h->kkt_valid) { kq_status rc = kkt_assemble(h); if (rc != KQ_OK) return rc; }
  KQ_CUDA(h, cudaMemcpyAsync(h->tmp, v, h->nkp * 8, cudaMemcpyDefault, h->stream));
  kq_status rc = pcg_apply(h, h->tmp, h->zref, precision, nullptr);
  if (rc != KQ_OK) return rc;
  KQ_CUDA(h, cudaMemcpyAsync(out, h->zref, h->nkp * 8, cudaMemcpyDefault, h->stream));
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  return KQ_OK;
}

kq_status kkt_pcg_solve(kq_handle h, const double *rhs, double *sol, const kq_pcg_opts *opts,
                        kq_pcg_stats *stats) {
  if (!h || !rhs || !sol) return kq_fail(h, KQ_ERR_ARG, "null argument");
  kq_pcg_opts o;
  kq_default_pcg_opts(&o);
  if (opts) o = *opts;
  if (!h->kkt_valid) { kq_status rc = kkt_assemble(h); if (rc != KQ_OK) return rc; }
  // rhs goes to K.rhs's sibling buffer: use acc arrays? use h->z as input copy
  double *rin = h->K.rhs;   // overwritten; the next assembly rebuilds it
  KQ_CUDA(h, cudaMemcpyAsync(rin, rhs, h->nkp * 8, cudaMemcpyDefault, h->stream));
  kq_status rc = pcg_solve(h, rin, h->z, o, stats);
  h->kkt_valid = false;
  if (rc != KQ_OK && rc != KQ_WARN_PCG_MAXIT) return rc;
  KQ_CUDA(h, cudaMemcpyAsync(sol, h->z, h->nkp * 8, cudaMemcpyDefault, h->stream));
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  return rc;
}

kq_status ipm_solve(kq_handle h, const kq_ipm_opts *opts, double *x, double *lam_lA,
                    double *lam_uA, double *lam_lx, double *lam_ux, double *lam_e,
                    kq_ipm_stats *stats) {
  if (!h) return kq_fail(nullptr, KQ_ERR_ARG, "null handle");
  auto t0 = std::chrono::steady_clock::now();
  const long long launches0 = h->launches;
  kq_status rc0;
  kq_ipm_opts o;
  kq_default_ipm_opts(&o);
  if (opts) o = *opts;
  h->timeout_s = o.timeout_s > 0 ? o.timeout_s : 2.0;
  kq_ipm_stats st{};
  kq_pcg_opts po;
  po.tol = o.pcg_tol; po.maxit = o.pcg_maxit; po.precision = o.precision;
  po.refine_steps = o.refine_steps; po.inner_tol = o.inner_tol;
  h->solved = false;
  double mu_start = o.mu0;
  if (h->state_set) {
    mu_start = h->mu;
    h->state_set = false;
  } else {
    if ((rc0 = init_state(h)) != KQ_OK) return rc0;
  }
  double mu = mu_start;
  int kexp = 0;
  h->mu = mu;
  double n2 = 0.0;
  kq_status rc = assemble_norms(h, &n2, nullptr);
  if (rc != KQ_OK) return rc;
  kq_status final = KQ_ERR_IPM_MAXIT;
  const DevProb &P = h->P;
  int it = 0;
  // Mixed precision pays where a product is bandwidth-bound.  Every mixed
  // Newton solve times its FP64 residual products; when an FP64 product costs
  // less than twice an FP32 iteration (a latency-bound problem, where FP32
  // passes only add iterations), the rest of the solve runs in FP64
  // (KQ_MIXED_SWITCH=0: never).
  bool to_f64 = false;
  const char *msw = getenv("KQ_MIXED_SWITCH");
  const bool allow_switch = !(msw && atoi(msw) == 0);
  h->record = o.record != 0;
  h->iter_log.clear();
  for (it = 1; it <= o.ipm_maxit; ++it) {
    kq_pcg_stats ps{};
    kq_ipm_iter rec{};
    if (h->record) {
      // max diag(K) / min diag(K) of this Newton system
      k_minmax<<<NB, NT, 0, h->stream>>>(h->nkp, h->K.diag, h->red);
      ++h->launches;
      double mm[2];
      if (fetch(h, 2, {1, 1}, mm) == KQ_OK && mm[0] > 0.0) rec.diag_ratio = -mm[1] / mm[0];
      rec.it = it;
      rec.mu = mu;
    }
    po.precision = to_f64 ? KQ_PREC_F64 : o.precision;
    h->warm_next = o.warm_start && it > 1;   // z holds the previous Newton direction
    rc = pcg_solve(h, h->K.rhs, h->z, po, &ps);
    if (h->record) {
      rec.pcg_iters = ps.iters;
      rec.pcg_iters_f64 = ps.iters_f64;
      rec.pcg_rel_res = ps.rel_res;
      rec.pcg_ms = ps.kernel_ms;
      rec.lanczos_steps = h->lz_steps;
      rec.lanczos_min = h->lz_min;
      rec.lanczos_max = h->lz_max;
      rec.kappa_jacobi = h->lz_min > 0.0 ? h->lz_max / h->lz_min : 0.0;
    }
    if (o.precision == KQ_PREC_MIXED && !to_f64 && allow_switch && ps.products_f64 > 0 &&
        ps.iters > ps.iters_f64) {
      const double t32 = (ps.kernel_ms - ps.kernel_ms_f64) / std::max(1, ps.iters - ps.iters_f64);
      const double t64 = ps.kernel_ms_f64 / std::max(1, ps.products_f64);
      if (t64 < 2.0 * t32) {
        to_f64 = true;
        st.switched_to_f64 = it;
      }
    }
    st.pcg_iters += ps.iters;
    st.pcg_kernel_ms += ps.kernel_ms;
    st.pcg_launches += 2 * ps.passes;
    st.pcg_products += ps.products;
    st.pcg_iters_f64 += ps.iters_f64;
    st.pcg_products_f64 += ps.products_f64;
    st.pcg_kernel_ms_f64 += ps.kernel_ms_f64;
    st.pcg_launches_f64 += ps.launches_f64;
    if (rc == KQ_WARN_PCG_MAXIT) st.pcg_maxit_hits++;
    else if (rc != KQ_OK) { final = rc; break; }
    // step recovery (A dx) and ratio test
    if ((rc = recover_enqueue(h)) != KQ_OK) { final = rc; break; }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) { final = kq_fail(h, KQ_ERR_CUDA, "sync"); break; }
    double ax, al;
    recover_finish(h, o.gamma, &ax, &al);
    if (!(ax == ax) || !(al == al)) { final = kq_fail(h, KQ_ERR_NUMERIC, "NaN step length"); break; }
    if ((rc = update_enqueue(h, ax, al)) != KQ_OK) { final = rc; break; }
    if ((rc = assemble_norms(h, &n2, nullptr)) != KQ_OK) { final = rc; break; }
    const double rn = sqrt(n2);
    if (!(rn == rn)) { final = kq_fail(h, KQ_ERR_NUMERIC, "residual norm is NaN"); break; }
    st.res_norm = rn;
    if (h->record) {
      rec.res_norm = rn;
      rec.primal_inf = sqrt(h->inf2[0]);
      rec.dual_inf = sqrt(h->inf2[1]);
      rec.compl_inf = sqrt(h->inf2[2]);
      rec.alpha_x = ax;
      rec.alpha_lam = al;
      h->iter_log.push_back(rec);
    }
    if (o.verbose)
      fprintf(stderr, "ipm %3d mu %.0e |r| %.3e ax %.4f al %.4f pcg %5d passes %d rel %.2e %.2f ms\n",
              it, mu, rn, ax, al, ps.iters, ps.passes, ps.rel_res, ps.kernel_ms);
    if (rn < mu) {
      if (mu < o.mu_tol) { final = KQ_OK; break; }
      ++kexp;
      mu = mu_start * pow(10.0, -(double)kexp);
      h->mu = mu;
      if ((rc = assemble_norms(h, &n2, nullptr)) != KQ_OK) { final = rc; break; }
    }
  }
  st.ipm_iters = std::min(it, o.ipm_maxit);
  st.mu_final = mu;
  st.status = final;
  if (final == KQ_OK) h->solved = true;
  // infeasibility norms of section 5.2 (scaled units) at the final iterate
  {
    double rH2 = 0.0;
    assemble_norms(h, &n2, &rH2);
    st.primal_inf = sqrt(h->inf2[0]);
    st.dual_inf = sqrt(rH2);
    st.compl_inf = sqrt(h->inf2[2]);
    st.res_norm = sqrt(n2);
  }
  // outputs
  const size_t nb = h->n * 8;
  if (x) cudaMemcpyAsync(x, h->S.x, nb, cudaMemcpyDefault, h->stream);
  if (lam_lA || lam_uA || lam_lx || lam_ux || lam_e) {
    double *olA = h->tmp + h->n + h->me, *ouA = h->tmp + h->n + h->me + h->m, *olx = h->acc2,
           *oux = h->acc3, *oe = h->tmp + h->n;
    k_unscale<<<NB, NT, 0, h->stream>>>(P, h->S, h->sigma, h->rhoC, olA, ouA,
                                         olx, oux, oe);
    if (lam_lA && h->m) cudaMemcpyAsync(lam_lA, olA, h->m * 8, cudaMemcpyDefault, h->stream);
    if (lam_uA && h->m) cudaMemcpyAsync(lam_uA, ouA, h->m * 8, cudaMemcpyDefault, h->stream);
    if (lam_lx) cudaMemcpyAsync(lam_lx, olx, nb, cudaMemcpyDefault, h->stream);
    if (lam_ux) cudaMemcpyAsync(lam_ux, oux, nb, cudaMemcpyDefault, h->stream);
    if (lam_e && h->me) cudaMemcpyAsync(lam_e, oe, h->me * 8, cudaMemcpyDefault, h->stream);
    h->kkt_valid = false;
  }
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  st.time_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  st.pcg_time_s = st.pcg_kernel_ms * 1e-3;
  st.kernel_launches = h->launches - launches0;
  if (stats) *stats = st;
  if (final == KQ_ERR_IPM_MAXIT) kq_fail(h, final, "IPM iteration cap reached");
  return final;
}

kq_status qp_backward(kq_handle h, const double *gbar, double *grad_p, double *grad_lA,
                      double *grad_uA, double *grad_b, const kq_pcg_opts *opts,
                      kq_pcg_stats *stats) {
  if (!h || !gbar) return kq_fail(h, KQ_ERR_ARG, "null argument");
  if (!h->solved) return kq_fail(h, KQ_ERR_STATE, "qp_backward needs a converged ipm_solve");
  kq_pcg_opts o;
  kq_default_pcg_opts(&o);
  if (opts) o = *opts;
  kq_status rc = kkt_assemble(h);   // K at the converged iterate and mu
  if (rc != KQ_OK) return rc;
  KQ_CUDA(h, cudaMemcpyAsync(h->tmp, gbar, h->n * 8, cudaMemcpyDefault, h->stream));
  k_pad_rhs<<<NB, NT, 0, h->stream>>>(h->nkp, h->tmp, h->n, h->K.rhs);
  ++h->launches;
  rc = pcg_solve(h, h->K.rhs, h->z, o, stats);
  h->kkt_valid = false;
  if (rc != KQ_OK && rc != KQ_WARN_PCG_MAXIT) return rc;
  double *gp = h->acc1, *glA = h->tmp + h->n + h->me, *guA = h->tmp + h->n + h->me + h->m,
         *gb = h->tmp + h->n;
  k_adjoint_out<<<NB, NT, 0, h->stream>>>(h->P, h->sigma, h->rhoC, h->z, gp,
                                           glA, guA, gb);
  if (grad_p) KQ_CUDA(h, cudaMemcpyAsync(grad_p, gp, h->n * 8, cudaMemcpyDefault, h->stream));
  if (grad_lA && h->m) KQ_CUDA(h, cudaMemcpyAsync(grad_lA, glA, h->m * 8, cudaMemcpyDefault, h->stream));
  if (grad_uA && h->m) KQ_CUDA(h, cudaMemcpyAsync(grad_uA, guA, h->m * 8, cudaMemcpyDefault, h->stream));
  if (grad_b && h->me) KQ_CUDA(h, cudaMemcpyAsync(grad_b, gb, h->me * 8, cudaMemcpyDefault, h->stream));
  KQ_CUDA(h, cudaStreamSynchronize(h->stream));
  return rc;
}

}  // extern "C"
