// kkt_pcg_solve_static: the persistent Jacobi-PCG solve of the doubly
// augmented KKT system for a dense problem, for callers that cannot allocate
// device memory (for example code that runs with a fixed, pre-reserved memory
// budget, or inside a framework whose allocator must not be bypassed).  All
// work space lives in one file-scope static device array of fixed size; the
// caller passes the problem blocks, the right-hand side and the solution
// buffer, all in device memory.
#include "common.cuh"
#include "kq_internal.h"
#include <atomic>
#include <cmath>
#include <string>

namespace {

// Limits of the static work space (documented in kktqp.h).
constexpr int64_t KQ_STATIC_MAX_N = 4096;
constexpr int64_t KQ_STATIC_MAX_M = 4096;
constexpr int KQ_STATIC_MAX_CTAS = 160;
constexpr int64_t KQ_STATIC_MAX_NKP = KQ_STATIC_MAX_N + 2 * KQ_STATIC_MAX_M;

// Doubles needed: 5 NKP vectors (r, y, p_old, p_new, diag), qlam (2m), accx (n),
// 5 per-row arrays (rho, cl, cu and the two bound flags packed as doubles),
// slots (4 per CTA), resn (2), plus 16 words of counters.
constexpr int64_t KQ_STATIC_DOUBLES = 5 * KQ_STATIC_MAX_NKP + 2 * KQ_STATIC_MAX_M +
                                      KQ_STATIC_MAX_N + 5 * KQ_STATIC_MAX_M +
                                      4 * KQ_STATIC_MAX_CTAS + 2 + 16;

// The scratch array: every GPU that loads the library holds it until exit
// (about 0.76 MB).  All calls share it.
static __device__ __align__(256) double g_kq_static_scratch[KQ_STATIC_DOUBLES];

// Device address of the array, looked up once per device (host code must not
// use the symbol itself: in host code it is only a stand-in).  Atomic so that
// host threads calling on different handles or streams read and publish it
// without a data race; two threads racing on the first call both look it up
// and store the same value.  Calls after cudaDeviceReset are not supported
// (the module is reloaded and the cached address is stale).
std::atomic<double *> g_scratch_addr[64];
thread_local std::string g_static_err;

// Jacobi diagonal of K (Eq. (9)) for dense H and A with all rows two-sided:
// diag_x = H_jj + dg_j + 2 sum_a A_aj^2 (1/Dl_a + 1/Du_a), diag_lam = (Dl, Du);
// also rho = 1, cl = 1/Dl, cu = 1/Du and both bound flags set.
__global__ void k_static_prep(int64_t n, int64_t m, const double *H, const double *A,
                              const double *Dl, const double *Du, const double *dg,
                              double *diag, double *rho, double *cl, double *cu,
                              uint8_t *hasl, uint8_t *hasu) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = tid; j < n; j += stride) {
    double s = 0.0;
    for (int64_t a = 0; a < m; ++a) {
      const double v = A[a * n + j];
      s += v * v * (1.0 / Dl[a] + 1.0 / Du[a]);
    }
    diag[j] = H[j * n + j] + dg[j] + 2.0 * s;
  }
  for (int64_t a = tid; a < m; a += stride) {
    diag[n + a] = Dl[a];
    diag[n + m + a] = Du[a];
    rho[a] = 1.0;
    cl[a] = 1.0 / Dl[a];
    cu[a] = 1.0 / Du[a];
    hasl[a] = 1;
    hasu[a] = 1;
  }
}

__global__ void k_static_check(int64_t m, const double *Dl, const double *Du, int *bad) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < m;
       a += (int64_t)gridDim.x * blockDim.x) {
    const double l = Dl[a], u = Du[a];
    if (!(l > 0.0) || !(u > 0.0) || isinf(l) || isinf(u)) atomicOr(bad, 1);
  }
}

}  // namespace

extern "C" kq_status kkt_pcg_solve_static(int64_t n, int64_t m, const double *H,
                                          const double *A, const double *Dl, const double *Du,
                                          const double *dg, const double *rhs, double *sol,
                                          double tol, int maxit, void *stream, int *iters,
                                          double *rel_res) {
  if (n <= 0 || m < 0 || n > KQ_STATIC_MAX_N || m > KQ_STATIC_MAX_M) {
    g_static_err = "kkt_pcg_solve_static: needs 0 < n <= 4096 and 0 <= m <= 4096";
    return kq_fail(nullptr, KQ_ERR_ARG, g_static_err);
  }
  if (!H || !dg || !rhs || !sol || (m > 0 && (!A || !Dl || !Du)) || maxit < 0 || !(tol >= 0.0))
    return kq_fail(nullptr, KQ_ERR_ARG, "kkt_pcg_solve_static: null pointer or bad tol/maxit");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return kq_fail(nullptr, KQ_ERR_CUDA, "kkt_pcg_solve_static: no current CUDA device");
  // one-time set-up on this device: the device address of the static array
  double *base = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!base) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_kq_static_scratch);
    if (e != cudaSuccess || !p)
      return kq_fail(nullptr, KQ_ERR_CUDA,
                     std::string("kkt_pcg_solve_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    base = static_cast<double *>(p);
    g_scratch_addr[dev].store(base, std::memory_order_release);
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return kq_fail(nullptr, KQ_ERR_CUDA, "kkt_pcg_solve_static: device query failed");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nkp = n + 2 * m;
  // carve the static array
  double *r = base, *y = r + nkp, *pb0 = y + nkp, *pb1 = pb0 + nkp, *diag = pb1 + nkp;
  double *qlam = diag + nkp, *accx = qlam + 2 * m, *rho = accx + n, *cl = rho + m, *cu = cl + m;
  uint8_t *hasl = reinterpret_cast<uint8_t *>(cu + m);   // m bytes
  uint8_t *hasu = hasl + m;                               // m bytes
  double *slots = cu + m + (2 * m + 7) / 8 + 1;           // after the 2m flag bytes
  double *resn = slots + 4 * KQ_STATIC_MAX_CTAS;
  unsigned int *bar = reinterpret_cast<unsigned int *>(resn + 2);
  int *err = reinterpret_cast<int *>(bar + 2);
  int *its = err + 1;
  int *bad = its + 1;
  // counters and flags start at zero on every call (the array keeps the last
  // call's contents)
  cudaError_t e = cudaMemsetAsync(bar, 0, 16 * sizeof(double), s);
  if (e != cudaSuccess)
    return kq_fail(nullptr, KQ_ERR_CUDA, std::string("kkt_pcg_solve_static: ") + cudaGetErrorString(e));
  if (m > 0) {
    k_static_check<<<32, 256, 0, s>>>(m, Dl, Du, bad);
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return kq_fail(nullptr, KQ_ERR_CUDA, "kkt_pcg_solve_static: check failed");
    if (hbad) return kq_fail(nullptr, KQ_ERR_ARG, "kkt_pcg_solve_static: Dl and Du must be finite and > 0");
  }
  k_static_prep<<<64, 256, 0, s>>>(n, m, H, A, Dl, Du, dg, diag, rho, cl, cu, hasl, hasu);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return kq_fail(nullptr, KQ_ERR_CUDA, std::string("kkt_pcg_solve_static: ") + cudaGetErrorString(e));
  DevProb P;
  P.n = n; P.m = m; P.me = 0; P.nkp = nkp;
  P.hkind = KQ_H_DENSE; P.hdtype = KQ_F64; P.hscale = 1.0;
  P.Hd = H; P.akind = m > 0 ? KQ_A_DENSE : KQ_A_NONE; P.adtype = KQ_F64; P.Ad = A;
  P.rhoA = rho; P.hasl = hasl; P.hasu = hasu;
  const int64_t rows = n + 2 * m;
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(sms, KQ_STATIC_MAX_CTAS),
                                                             ceil_div64(rows, 32)));
  PcgRawWork w{r, y, pb0, pb1, qlam, slots, resn, accx, bar, err, its};
  int it = 0;
  double rr = 0.0, bb = 0.0;
  std::string msg;
  const kq_status st = pcg_dense_raw(P, Dl, Du, cl, cu, dg, diag, rhs, sol, w, G, tol, maxit, 2.0, s,
                                     &it, &rr, &bb, &msg);
  if (iters) *iters = it;
  if (rel_res) *rel_res = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  if (st != KQ_OK) return kq_fail(nullptr, st, "kkt_pcg_solve_static: " + msg);
  if (bb > 0.0 && rr > tol * tol * bb) return KQ_WARN_PCG_MAXIT;
  return KQ_OK;
}
