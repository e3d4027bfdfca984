// FP64 CPU implementation of the 2x2 direction-independent calibration, all host cores (OpenMP):
// StefCal (Sect. 4.3 eq. update:DI:diag:pol with the product order [sum D Y^H][sum Y Y^H]^-1 and the
// GN / average alternation of Sect. 3.1) followed by App. C's Levenberg-Marquardt with the whole
// J^H J of Sect. 4.2 eq. JHJ:pol.  It is the timed CPU comparator of the benchmark.
//
// TEST AND BENCHMARK INFRASTRUCTURE ONLY: it shares no code with the CUDA library (it is compiled
// on its own and loaded by the benchmark's CPU leg), and nothing on the product path calls it.
//
// One interval per OpenMP task.  Per interval the gains do not depend on the sample, so the sample
// sums are taken once (Sect. 3.2.1: gains factor out of the sums over s), in FP64:
//   P_b = sum_s conj(M) (x) D          (vec(D G_q M^H) = P_b vec G_q; (x) the Kronecker product)
//   F_b = sum_s conj(M) (x) M          (vec(M X M^H) = F_b vec X)
//   E_b = sum_s ||D||^2
// vec stacks columns (App. B).  Unknowns of the LM step: the real and imaginary parts of vec G_p per
// antenna, n = 8 N_ant; the step solves (H + lambda diag H + mu v v^T) x = (I - v v^T) g with v the
// phase-gauge direction i G / ||G|| and mu the mean of diag H (see the GPU header for the same
// reading), by an FP64 Cholesky factorisation.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include <omp.h>

namespace {

using cd = std::complex<double>;

struct Mom {
  cd P[16];   // row-major 4x4
  cd F[16];
  double E;
};

inline void vecm(const cd* G, cd* v) { v[0] = G[0]; v[1] = G[2]; v[2] = G[1]; v[3] = G[3]; }  // G row-major
inline void unvec(const cd* v, cd* G) { G[0] = v[0]; G[2] = v[1]; G[1] = v[2]; G[3] = v[3]; }
inline void mv4(const cd* A, const cd* x, cd* y) {
  for (int r = 0; r < 4; ++r) { cd s = 0; for (int k = 0; k < 4; ++k) s += A[r * 4 + k] * x[k]; y[r] = s; }
}
inline void mhv4(const cd* A, const cd* x, cd* y) {  // A^H x
  for (int k = 0; k < 4; ++k) { cd s = 0; for (int r = 0; r < 4; ++r) s += std::conj(A[r * 4 + k]) * x[r]; y[k] = s; }
}
inline void mm2(const cd* A, const cd* B, cd* C) {  // row-major 2x2
  C[0] = A[0] * B[0] + A[1] * B[2]; C[1] = A[0] * B[1] + A[1] * B[3];
  C[2] = A[2] * B[0] + A[3] * B[2]; C[3] = A[2] * B[1] + A[3] * B[3];
}
inline void hmm2(const cd* A, const cd* B, cd* C) {  // A^H B
  C[0] = std::conj(A[0]) * B[0] + std::conj(A[2]) * B[2]; C[1] = std::conj(A[0]) * B[1] + std::conj(A[2]) * B[3];
  C[2] = std::conj(A[1]) * B[0] + std::conj(A[3]) * B[2]; C[3] = std::conj(A[1]) * B[1] + std::conj(A[3]) * B[3];
}
// Phi(X) = sum_s M X M^H through F; Phi'(X) = sum_s M^H X M through F^H
inline void phi(const Mom& m, const cd* X, cd* Y, bool adj) {
  cd v[4], w[4];
  vecm(X, v);
  if (adj) mhv4(m.F, v, w); else mv4(m.F, v, w);
  unvec(w, Y);
}

struct Interval {
  int n_ant, n_bl;
  const int32_t* a1;
  const int32_t* a2;
  std::vector<Mom> mom;
};

void moments(const float* vis, const float* model, int64_t r0, int ns, Interval& iv) {
  iv.mom.assign(iv.n_bl, Mom{});
  for (int b = 0; b < iv.n_bl; ++b) {
    Mom& m = iv.mom[b];
    for (int s = 0; s < ns; ++s) {
      const int64_t row = r0 + (int64_t)s * iv.n_bl + b;
      cd D[4], M[4];
      for (int e = 0; e < 4; ++e) {
        D[e] = cd(vis[8 * row + 2 * e], vis[8 * row + 2 * e + 1]);
        M[e] = cd(model[8 * row + 2 * e], model[8 * row + 2 * e + 1]);
      }
      // kron(conj M, X)[2 i1 + i2][2 j1 + j2] = conj(M[i1][j1]) X[i2][j2]
      for (int i1 = 0; i1 < 2; ++i1)
        for (int i2 = 0; i2 < 2; ++i2)
          for (int j1 = 0; j1 < 2; ++j1)
            for (int j2 = 0; j2 < 2; ++j2) {
              const cd cm = std::conj(M[2 * i1 + j1]);
              m.P[(2 * i1 + i2) * 4 + 2 * j1 + j2] += cm * D[2 * i2 + j2];
              m.F[(2 * i1 + i2) * 4 + 2 * j1 + j2] += cm * M[2 * i2 + j2];
            }
      for (int e = 0; e < 4; ++e) m.E += std::norm(D[e]);
    }
  }
}

// per antenna: C = sum D Y^H (top half of J^H D) and Hb = sum Y Y^H, at gains G
void blocks(const Interval& iv, const std::vector<cd>& G, std::vector<cd>& C, std::vector<cd>& Hb) {
  C.assign(4 * iv.n_ant, 0.0);
  Hb.assign(4 * iv.n_ant, 0.0);
  for (int b = 0; b < iv.n_bl; ++b) {
    const int p = iv.a1[b], q = iv.a2[b];
    const Mom& m = iv.mom[b];
    cd v[4], w[4], X[4], Y[4], A[4];
    vecm(&G[4 * q], v); mv4(m.P, v, w); unvec(w, X);                 // sum D G_q M^H
    for (int e = 0; e < 4; ++e) C[4 * p + e] += X[e];
    hmm2(&G[4 * q], &G[4 * q], A); phi(m, A, Y, false);             // sum M G_q^H G_q M^H
    for (int e = 0; e < 4; ++e) Hb[4 * p + e] += Y[e];
    vecm(&G[4 * p], v); mhv4(m.P, v, w); unvec(w, X);                // sum D^H G_p M
    for (int e = 0; e < 4; ++e) C[4 * q + e] += X[e];
    hmm2(&G[4 * p], &G[4 * p], A); phi(m, A, Y, true);              // sum M^H G_p^H G_p M
    for (int e = 0; e < 4; ++e) Hb[4 * q + e] += Y[e];
  }
}

double chi2(const Interval& iv, const std::vector<cd>& G) {
  double c = 0;
  for (int b = 0; b < iv.n_bl; ++b) {
    const int p = iv.a1[b], q = iv.a2[b];
    const Mom& m = iv.mom[b];
    cd vp[4], vq[4], w[4], A[4], Ap[4], Y[4];
    vecm(&G[4 * p], vp); vecm(&G[4 * q], vq); mv4(m.P, vq, w);
    cd t2 = 0;
    for (int r = 0; r < 4; ++r) t2 += std::conj(vp[r]) * w[r];
    hmm2(&G[4 * q], &G[4 * q], A); phi(m, A, Y, false); hmm2(&G[4 * p], &G[4 * p], Ap);
    cd t3 = 0;   // tr(G_p^H G_p Y)
    for (int i = 0; i < 2; ++i)
      for (int k = 0; k < 2; ++k) t3 += Ap[i * 2 + k] * Y[k * 2 + i];
    c += m.E - 2.0 * t2.real() + t3.real();
  }
  return c;
}

inline bool inv2(const cd* H, cd* Hi) {
  const cd det = H[0] * H[3] - H[1] * H[2];
  if (!(std::abs(det) > 0)) return false;
  Hi[0] = H[3] / det; Hi[1] = -H[1] / det; Hi[2] = -H[2] / det; Hi[3] = H[0] / det;
  return true;
}

// Real form of the map d -> d A (A 2x2 complex) on the real coordinates of one antenna:
// index 2 * (2 r + c) + {0: re, 1: im} of entry (r, c) of d (row-major).
inline void add_right_mult(const cd* A, double* Hm, int ld, int row0, int col0) {
  for (int r = 0; r < 2; ++r)
    for (int c_out = 0; c_out < 2; ++c_out)
      for (int c_in = 0; c_in < 2; ++c_in) {
        const cd t = A[c_in * 2 + c_out];   // (d A)[r][c_out] += d[r][c_in] A[c_in][c_out]
        const int o = row0 + 2 * (2 * r + c_out), i = col0 + 2 * (2 * r + c_in);
        Hm[(size_t)o * ld + i] += t.real();       Hm[(size_t)o * ld + i + 1] -= t.imag();
        Hm[(size_t)(o + 1) * ld + i] += t.imag(); Hm[(size_t)(o + 1) * ld + i + 1] += t.real();
      }
}

// Whole GN matrix (real, n = 8 N) and gradient J^H R at G.  Cross block for baseline (p, q):
// d_q -> G_p Phi(d_q^H G_q), and its transpose for (q, p).
void assemble(const Interval& iv, const std::vector<cd>& G, std::vector<double>& Hm, std::vector<double>& g) {
  const int N = iv.n_ant, n = 8 * N;
  Hm.assign((size_t)n * n, 0.0);
  g.assign(n, 0.0);
  std::vector<cd> C, Hb;
  blocks(iv, G, C, Hb);
  for (int p = 0; p < N; ++p) {
    cd GH[4];
    mm2(&G[4 * p], &Hb[4 * p], GH);
    for (int e = 0; e < 4; ++e) {
      const cd d = C[4 * p + e] - GH[e];
      g[8 * p + 2 * e] = d.real(); g[8 * p + 2 * e + 1] = d.imag();
    }
    add_right_mult(&Hb[4 * p], Hm.data(), n, 8 * p, 8 * p);
  }
  for (int b = 0; b < iv.n_bl; ++b) {
    const int p = iv.a1[b], q = iv.a2[b];
    const Mom& m = iv.mom[b];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int h = 0; h < 2; ++h) {   // d_q = E_ij (h = 0) or i E_ij (h = 1)
          cd X[4] = {0, 0, 0, 0};        // d_q^H G_q: row j = conj(c) * row i of G_q
          const cd cc = h ? cd(0, -1) : cd(1, 0);
          X[2 * j + 0] = cc * G[4 * q + 2 * i + 0];
          X[2 * j + 1] = cc * G[4 * q + 2 * i + 1];
          cd Y[4], Z[4];
          phi(m, X, Y, false);
          mm2(&G[4 * p], Y, Z);
          const int col = 8 * q + 2 * (2 * i + j) + h;
          for (int e = 0; e < 4; ++e) {
            const int row = 8 * p + 2 * e;
            Hm[(size_t)row * n + col] += Z[e].real();
            Hm[(size_t)(row + 1) * n + col] += Z[e].imag();
            Hm[(size_t)col * n + row] += Z[e].real();        // the (q, p) block is the transpose
            Hm[(size_t)col * n + row + 1] += Z[e].imag();
          }
        }
  }
}

// In-place Cholesky (lower) and solve; false if a pivot is not positive.
bool chol_solve(std::vector<double>& A, int n, std::vector<double>& x) {
  for (int k = 0; k < n; ++k) {
    double* rk = &A[(size_t)k * n];
    double d = rk[k];
    for (int t = 0; t < k; ++t) d -= rk[t] * rk[t];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    rk[k] = d;
    const double inv = 1.0 / d;
    for (int i = k + 1; i < n; ++i) {
      double* ri = &A[(size_t)i * n];
      double s = ri[k];
      for (int t = 0; t < k; ++t) s -= ri[t] * rk[t];
      ri[k] = s * inv;
    }
  }
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int t = 0; t < i; ++t) s -= A[(size_t)i * n + t] * x[t];
    x[i] = s / A[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int t = i + 1; t < n; ++t) s -= A[(size_t)t * n + i] * x[t];
    x[i] = s / A[(size_t)i * n + i];
  }
  return true;
}

int solve_interval(Interval& iv, std::vector<cd>& G, double tol, int max_iter, int lm_after, double lam0, double K,
                   int* iters) {
  const int N = iv.n_ant, n = 8 * N;
  int k = 0;
  // StefCal: odd k GN, even k average
  for (; k < lm_after && k < max_iter; ++k) {
    std::vector<cd> C, Hb;
    blocks(iv, G, C, Hb);
    std::vector<cd> Gn(G);
    for (int p = 0; p < N; ++p) {
      cd Hi[4];
      if (!inv2(&Hb[4 * p], Hi)) continue;
      mm2(&C[4 * p], Hi, &Gn[4 * p]);
    }
    if ((k + 1) % 2 == 0)
      for (size_t e = 0; e < G.size(); ++e) Gn[e] = 0.5 * (G[e] + Gn[e]);
    G.swap(Gn);
  }
  // LM
  double lam = lam0, chi = chi2(iv, G);
  std::vector<double> Hm, g, A, x;
  int status = 1;
  for (; k < max_iter; ++k) {
    assemble(iv, G, Hm, g);
    double dsum = 0, gn2 = 0;
    for (int e = 0; e < n; ++e) dsum += Hm[(size_t)e * n + e];
    for (auto& z : G) gn2 += std::norm(z);
    const double mu = dsum / n, vn = 1.0 / std::sqrt(gn2);
    std::vector<double> v(n);
    for (int e = 0; e < n / 2; ++e) { v[2 * e] = -G[e].imag() * vn; v[2 * e + 1] = G[e].real() * vn; }
    double vg = 0;
    for (int e = 0; e < n; ++e) vg += v[e] * g[e];
    x.resize(n);
    for (int e = 0; e < n; ++e) x[e] = g[e] - v[e] * vg;
    A = Hm;
    for (int r = 0; r < n; ++r) {
      A[(size_t)r * n + r] += lam * Hm[(size_t)r * n + r];
      for (int c = 0; c < n; ++c) A[(size_t)r * n + c] += mu * v[r] * v[c];
    }
    if (!chol_solve(A, n, x)) { lam *= K; continue; }
    std::vector<cd> Gt(G);
    double dx2 = 0, gt2 = 0;
    for (int e = 0; e < n / 2; ++e) {
      Gt[e] += cd(x[2 * e], x[2 * e + 1]);
      dx2 += x[2 * e] * x[2 * e] + x[2 * e + 1] * x[2 * e + 1];
      gt2 += std::norm(Gt[e]);
    }
    const double ct = chi2(iv, Gt);
    const bool acc = ct < chi;
    if (acc) { G.swap(Gt); chi = ct; lam /= K; } else lam *= K;
    if (dx2 <= tol * tol * gt2) { status = 0; ++k; break; }
  }
  *iters = k;
  return status;
}

}  // namespace

extern "C" {

// vis, model: complex64 2x2 rows; gains: complex64 2x2 per antenna (in: start, out: solution).
// Layout as gc_layout (host arrays).  Returns the number of threads used.
int cpu_calibrate_jones_lm(const float* vis, const float* model, int n_int, const int64_t* row_off,
                           const int32_t* n_samp, const int32_t* n_bl, const int32_t* bl_off, const int32_t* n_ant,
                           const int32_t* gain_off, const int32_t* ant1, const int32_t* ant2, float* gains, double tol,
                           int max_iter, int lm_after, double lam0, double K, int32_t* iters, int32_t* status,
                           int n_threads) {
  if (n_threads > 0) omp_set_num_threads(n_threads);
  int used = 1;
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < n_int; ++i) {
      Interval iv;
      iv.n_ant = n_ant[i];
      iv.n_bl = n_bl[i];
      iv.a1 = ant1 + bl_off[i];
      iv.a2 = ant2 + bl_off[i];
      moments(vis, model, row_off[i], n_samp[i], iv);
      std::vector<cd> G(4 * iv.n_ant);
      float* gp = gains + (size_t)8 * gain_off[i];
      for (int e = 0; e < 4 * iv.n_ant; ++e) G[e] = cd(gp[2 * e], gp[2 * e + 1]);
      int it = 0;
      status[i] = solve_interval(iv, G, tol, max_iter, lm_after, lam0, K, &it);
      iters[i] = it;
      for (int e = 0; e < 4 * iv.n_ant; ++e) { gp[2 * e] = (float)G[e].real(); gp[2 * e + 1] = (float)G[e].imag(); }
    }
  }
  return used;
}

}  // extern "C"
