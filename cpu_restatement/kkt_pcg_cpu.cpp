// CPU restatement of the paper's own Newton-step design (section 3.2): the
// doubly augmented KKT system of Eq. (9), K = [Q + 2B'D^-1B, B'; B, D] with
// Q = H + diag(dg) and B = [A_L; -A_U], applied matrix-free from H = P' W2 P
// (P CSR, W2 = diag(w2)), A, A' and D, and solved by Jacobi-preconditioned CG
// (stop when |rhs - K z|_2 <= tol |rhs|_2, z0 = 0).  FP64 throughout, OpenMP
// over rows; the transposed products accumulate into one private n-vector
// per thread, summed afterwards.
//
// A measurement baseline for the CPU side, the analogue of the paper's
// C++/OpenBLAS prototype (section 4): it shares no code with the GPU library
// or the oracle.  Structures covered: the CSR least-squares Hessian with
// general CSR rows (no equality rows), i.e. the dose QPs.
#include <omp.h>
#include <stdint.h>
#include <string.h>
#include <math.h>
#include <vector>

namespace {

struct Sys {
  int64_t n, nP, m;
  const int64_t *prow; const int32_t *pcol; const double *pval; const double *w2;
  const int64_t *arow; const int32_t *acol; const double *aval;
  int64_t nl, nu; const int32_t *L; const int32_t *U;   // rows of A with a lower / upper bound
  const double *dg, *D;                                  // D: nl + nu entries (L rows, then U rows)
};

// out = K v (length n + nl + nu); scratch: Pv (nP), Av (m), z (m), per-thread n-vectors
void apply(const Sys &S, const double *v, double *out, std::vector<double> &Pv,
           std::vector<double> &Av, std::vector<double> &z, std::vector<double> &acc) {
  const int64_t n = S.n, nl = S.nl, nu = S.nu;
  const double *vx = v, *vl = v + n;
  const int nth = omp_get_max_threads();
#pragma omp parallel
  {
#pragma omp for schedule(static)
    for (int64_t r = 0; r < S.nP; ++r) {
      double s = 0.0;
      for (int64_t k = S.prow[r]; k < S.prow[r + 1]; ++k) s += S.pval[k] * vx[S.pcol[k]];
      Pv[r] = S.w2[r] * s;
    }
#pragma omp for schedule(static)
    for (int64_t i = 0; i < S.m; ++i) {
      double s = 0.0;
      for (int64_t k = S.arow[i]; k < S.arow[i + 1]; ++k) s += S.aval[k] * vx[S.acol[k]];
      Av[i] = s;
      z[i] = 0.0;
    }
    // t = B v_x; bottom = t + D v_l; z = A'-weights of 2 t / D + v_l
#pragma omp for schedule(static)
    for (int64_t j = 0; j < nl; ++j) {
      const double t = Av[S.L[j]];
      out[n + j] = t + S.D[j] * vl[j];
      z[S.L[j]] += 2.0 * t / S.D[j] + vl[j];
    }
#pragma omp barrier
#pragma omp for schedule(static)
    for (int64_t j = 0; j < nu; ++j) {
      const double t = -Av[S.U[j]];
      out[n + nl + j] = t + S.D[nl + j] * vl[nl + j];
      z[S.U[j]] -= 2.0 * t / S.D[nl + j] + vl[nl + j];
    }
    // top = P'(W2 P v) + A' z + dg v, each thread into its own n-vector
    const int t = omp_get_thread_num();
    double *a = acc.data() + (size_t)t * n;
    for (int64_t c = 0; c < n; ++c) a[c] = 0.0;
#pragma omp for schedule(static)
    for (int64_t r = 0; r < S.nP; ++r) {
      const double u = Pv[r];
      for (int64_t k = S.prow[r]; k < S.prow[r + 1]; ++k) a[S.pcol[k]] += S.pval[k] * u;
    }
#pragma omp for schedule(static)
    for (int64_t i = 0; i < S.m; ++i) {
      const double u = z[i];
      if (u != 0.0)
        for (int64_t k = S.arow[i]; k < S.arow[i + 1]; ++k) a[S.acol[k]] += S.aval[k] * u;
    }
#pragma omp for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      double s = S.dg[c] * vx[c];
      for (int th = 0; th < nth; ++th) s += acc[(size_t)th * n + c];
      out[c] = s;
    }
  }
}

double dot(int64_t N, const double *a, const double *b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < N; ++i) s += a[i] * b[i];
  return s;
}

}  // namespace

extern "C" {

// K v of Eq. (9).  L, U: rows of A with a finite lower / upper limit (D holds
// their entries in that order); v and out have n + nl + nu entries.
int cpu_kkt_apply(int64_t n, int64_t nP, const int64_t *prow, const int32_t *pcol,
                  const double *pval, const double *w2, int64_t m, const int64_t *arow,
                  const int32_t *acol, const double *aval, int64_t nl, const int32_t *L,
                  int64_t nu, const int32_t *U, const double *dg, const double *D,
                  const double *v, double *out) {
  Sys S{n, nP, m, prow, pcol, pval, w2, arow, acol, aval, nl, nu, L, U, dg, D};
  std::vector<double> Pv(nP), Av(m), z(m), acc((size_t)omp_get_max_threads() * n);
  apply(S, v, out, Pv, Av, z, acc);
  return 0;
}

// Jacobi-PCG on Eq. (9): z0 = 0, stop when |r|_2 <= tol |rhs|_2 or after
// maxit iterations (tol = 0: exactly maxit).  Returns the iterations taken;
// *rel = |r|_2 / |rhs|_2 of the recurrence residual at exit.
int cpu_kkt_pcg(int64_t n, int64_t nP, const int64_t *prow, const int32_t *pcol,
                const double *pval, const double *w2, int64_t m, const int64_t *arow,
                const int32_t *acol, const double *aval, int64_t nl, const int32_t *L,
                int64_t nu, const int32_t *U, const double *dg, const double *D,
                const double *diag, const double *rhs, double tol, int maxit, double *sol,
                double *rel) {
  Sys S{n, nP, m, prow, pcol, pval, w2, arow, acol, aval, nl, nu, L, U, dg, D};
  const int64_t N = n + nl + nu;
  std::vector<double> Pv(nP), Av(m), zz(m), acc((size_t)omp_get_max_threads() * n);
  std::vector<double> r(rhs, rhs + N), y(N), p(N), q(N);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    sol[i] = 0.0;
    y[i] = r[i] / diag[i];
    p[i] = y[i];
  }
  const double bn = sqrt(dot(N, rhs, rhs));
  double rho = dot(N, r.data(), y.data()), rn = bn;
  int it = 0;
  while (it < maxit && !(rn <= tol * bn)) {
    apply(S, p.data(), q.data(), Pv, Av, zz, acc);
    const double pq = dot(N, p.data(), q.data());
    if (!(pq > 0.0)) break;
    const double alpha = rho / pq;
    double rr = 0.0, ry = 0.0;
#pragma omp parallel for reduction(+ : rr, ry) schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      sol[i] += alpha * p[i];
      r[i] -= alpha * q[i];
      y[i] = r[i] / diag[i];
      rr += r[i] * r[i];
      ry += r[i] * y[i];
    }
    const double beta = ry / rho;
    rho = ry;
    rn = sqrt(rr);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) p[i] = y[i] + beta * p[i];
    ++it;
  }
  if (rel) *rel = bn > 0.0 ? rn / bn : 0.0;
  return it;
}

int cpu_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
