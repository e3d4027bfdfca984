// Per-kind arithmetic of the direction-independent solvers (scalar gains and 2x2 Jones), shared by
// the streaming kernels (di_kernels.cu) and the moment / resident kernels (resident.cu).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace gc {

template <typename T> GC_DEV M2<T> scale_m2(M2<T> x, T s) {
  x.a = scale_(x.a, s); x.b = scale_(x.b, s); x.c = scale_(x.c, s); x.d = scale_(x.d, s);
  return x;
}
// sqrt of row r's weight (Sect. 2.4, a diagonal W), 1 without weights
template <typename T> GC_DEV T row_sw(const T* w, int64_t r) { return w ? sqrt(w[r]) : T(1); }
// row r's weight, 1 without weights
template <typename T> GC_DEV T row_w(const T* w, int64_t r) { return w ? w[r] : T(1); }

// ------------------------------------------------------------------------------------------
// Per-kind row arithmetic.  Partial-sum component order (per side):
//   scalar: [Re c, Im c, A]                              c = sum conj(y) d, A = sum |y|^2
//   jones : [C00, C01, C10, C11 (re,im each), H00, H11, Re H01, Im H01]
//           C = sum D Y^H, H = sum Y Y^H
// ------------------------------------------------------------------------------------------
template <typename T>
struct ScalarKind {
  static constexpr int NC = 3;  // components per side
  static constexpr int GW = 2;  // reals per gain
  using G = Cx<T>;
  static GC_DEV G ld_gain(const T* g) { return cx<T>(g[0], g[1]); }
  static GC_DEV void st_gain(T* g, const G& v) { g[0] = v.x; g[1] = v.y; }

  // Row (p, q, s): y = m conj(g_q) feeds antenna p; the conjugate row (q, p) has
  // y_qp = conj(m) conj(g_p) = conj(w) with w = g_p m and d_qp = conj(d).  sw = sqrt of the row's
  // weight (Sect. 2.4): d and m scaled by it make every sum below carry the weight once.
  static GC_DEV void row(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq, T* pp, T* pq, T sw) {
    const Cx<T> d = scale_(Vec<T>::ld1(vis + 2 * r), sw);
    const Cx<T> m = scale_(Vec<T>::ld1(mod + 2 * r), sw);
    const Cx<T> y = mulc_(m, gq);
    const Cx<T> w = mul_(gp, m);
    pp[0] = fma(y.x, d.x, fma(y.y, d.y, pp[0]));   // conj(y) d
    pp[1] = fma(y.x, d.y, fma(-y.y, d.x, pp[1]));
    pp[2] = fma(y.x, y.x, fma(y.y, y.y, pp[2]));
    pq[0] = fma(w.x, d.x, fma(w.y, d.y, pq[0]));   // w conj(d)
    pq[1] = fma(w.y, d.x, fma(-w.x, d.y, pq[1]));
    pq[2] = fma(w.x, w.x, fma(w.y, w.y, pq[2]));
  }

  // |d - g_p m conj(g_q)|^2
  static GC_DEV T resid2(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq) {
    const Cx<T> d = Vec<T>::ld1(vis + 2 * r);
    const Cx<T> m = Vec<T>::ld1(mod + 2 * r);
    const Cx<T> v = mulc_(mul_(gp, m), gq);
    return abs2_(sub_(d, v));
  }

  // GN gain from the sums; returns false (and leaves out = old) when A is not positive.
  static GC_DEV bool solve(const T* v, const G& old, G& out) {
    const T A = v[2];
    if (!(A > T(0))) { out = old; return false; }
    const T inv = T(1) / A;
    out = cx<T>(v[0] * inv, v[1] * inv);
    return true;
  }
  // sum over the antenna's rows of |d - g y|^2 - |d|^2 = A |g|^2 - 2 Re(conj(g) c), from its sums at g
  static GC_DEV double energy(const T* v, const G& g) {
    const double gx = g.x, gy = g.y;
    return (double)v[2] * (gx * gx + gy * gy) - 2.0 * ((double)v[0] * gx + (double)v[1] * gy);
  }
  static GC_DEV G avg(const G& a, const G& b) { return cx<T>(T(0.5) * (a.x + b.x), T(0.5) * (a.y + b.y)); }
  static GC_DEV T dist2(const G& a, const G& b) { return abs2_(sub_(a, b)); }
  static GC_DEV T norm2(const G& a) { return abs2_(a); }
  static GC_DEV bool finite(const G& a) { return isfinite(a.x) && isfinite(a.y); }
  static GC_DEV void write_acc(const T* v, T* jhd, T* jhj, int64_t slot) {
    jhd[2 * slot] = v[0]; jhd[2 * slot + 1] = v[1]; jhj[slot] = v[2];
  }
};

template <typename T>
struct JonesKind {
  static constexpr int NC = 12;
  static constexpr int GW = 8;
  using G = M2<T>;
  static GC_DEV G ld_gain(const T* g) {
    G m;
    m.a = cx<T>(g[0], g[1]); m.b = cx<T>(g[2], g[3]); m.c = cx<T>(g[4], g[5]); m.d = cx<T>(g[6], g[7]);
    return m;
  }
  static GC_DEV void st_gain(T* g, const G& m) {
    g[0] = m.a.x; g[1] = m.a.y; g[2] = m.b.x; g[3] = m.b.y;
    g[4] = m.c.x; g[5] = m.c.y; g[6] = m.d.x; g[7] = m.d.y;
  }

  // Row (p, q, s) with Y = M G_q^H feeds antenna p: C_p += D Y^H, H_p += Y Y^H.
  // Its conjugate row (q, p) has Y_qp = M^H G_p^H = W^H with W = G_p M and D_qp = D^H:
  //   C_q += D^H W,  H_q += W^H W.  sw: sqrt of the row's weight, applied to D and M.
  static GC_DEV void row(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq, T* pp, T* pq, T sw) {
    const M2<T> D = scale_m2(Vec<T>::ld4(vis + 8 * r), sw);
    const M2<T> M = scale_m2(Vec<T>::ld4(mod + 8 * r), sw);
    const M2<T> Y = mmh_(M, gq);
    const M2<T> W = mm_(gp, M);
    // p side
    fmac2(pp[0], pp[1], D.a, Y.a); fmac2(pp[0], pp[1], D.b, Y.b);
    fmac2(pp[2], pp[3], D.a, Y.c); fmac2(pp[2], pp[3], D.b, Y.d);
    fmac2(pp[4], pp[5], D.c, Y.a); fmac2(pp[4], pp[5], D.d, Y.b);
    fmac2(pp[6], pp[7], D.c, Y.c); fmac2(pp[6], pp[7], D.d, Y.d);
    pp[8] += abs2_(Y.a) + abs2_(Y.b);
    pp[9] += abs2_(Y.c) + abs2_(Y.d);
    fmac2(pp[10], pp[11], Y.a, Y.c); fmac2(pp[10], pp[11], Y.b, Y.d);
    // q side
    cfma2(pq[0], pq[1], D.a, W.a); cfma2(pq[0], pq[1], D.c, W.c);
    cfma2(pq[2], pq[3], D.a, W.b); cfma2(pq[2], pq[3], D.c, W.d);
    cfma2(pq[4], pq[5], D.b, W.a); cfma2(pq[4], pq[5], D.d, W.c);
    cfma2(pq[6], pq[7], D.b, W.b); cfma2(pq[6], pq[7], D.d, W.d);
    pq[8] += abs2_(W.a) + abs2_(W.c);
    pq[9] += abs2_(W.b) + abs2_(W.d);
    cfma2(pq[10], pq[11], W.a, W.b); cfma2(pq[10], pq[11], W.c, W.d);
  }

  // ||D - G_p M G_q^H||_F^2
  static GC_DEV T resid2(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq) {
    const M2<T> D = Vec<T>::ld4(vis + 8 * r);
    const M2<T> M = Vec<T>::ld4(mod + 8 * r);
    const M2<T> V = mmh_(mm_(gp, M), gq);
    return abs2_(sub_(D.a, V.a)) + abs2_(sub_(D.b, V.b)) + abs2_(sub_(D.c, V.c)) + abs2_(sub_(D.d, V.d));
  }

  // G = C H^-1 with H = [[h00, h01], [conj h01, h11]]; false when det(H) is not positive.
  static GC_DEV bool solve(const T* v, const G& old, G& out) {
    const T h00 = v[8], h11 = v[9];
    const Cx<T> h01 = cx<T>(v[10], v[11]);
    const T det = h00 * h11 - abs2_(h01);
    if (!(det > T(0)) || !(h00 > T(0))) { out = old; return false; }
    const T inv = T(1) / det;
    const Cx<T> C00 = cx<T>(v[0], v[1]), C01 = cx<T>(v[2], v[3]), C10 = cx<T>(v[4], v[5]), C11 = cx<T>(v[6], v[7]);
    // [C00 C01; C10 C11] [h11 -h01; -conj(h01) h00] / det
    out.a = scale_(sub_(scale_(C00, h11), mulc_(C01, h01)), inv);
    out.b = scale_(sub_(scale_(C01, h00), mul_(C00, h01)), inv);
    out.c = scale_(sub_(scale_(C10, h11), mulc_(C11, h01)), inv);
    out.d = scale_(sub_(scale_(C11, h00), mul_(C10, h01)), inv);
    return true;
  }
  // sum over the antenna's rows of ||D - G Y||^2 - ||D||^2 = tr(G H G^H) - 2 Re tr(C G^H), from its
  // sums at G (each row (x, y) of G adds h00 |x|^2 + h11 |y|^2 + 2 Re(x h01 conj(y)))
  static GC_DEV double energy(const T* v, const G& g) {
    const double h00 = v[8], h11 = v[9], hr = v[10], hi = v[11];
    auto row = [&](const Cx<T>& x, const Cx<T>& y) {
      const double xr = x.x, xi = x.y, yr = y.x, yi = y.y;
      // x h01 conj(y): real part of (xr + i xi)(hr + i hi)(yr - i yi)
      const double ar = xr * hr - xi * hi, ai = xr * hi + xi * hr;
      return h00 * (xr * xr + xi * xi) + h11 * (yr * yr + yi * yi) + 2.0 * (ar * yr + ai * yi);
    };
    const double gh = row(g.a, g.b) + row(g.c, g.d);
    const double cg = (double)v[0] * g.a.x + (double)v[1] * g.a.y + (double)v[2] * g.b.x + (double)v[3] * g.b.y +
                      (double)v[4] * g.c.x + (double)v[5] * g.c.y + (double)v[6] * g.d.x + (double)v[7] * g.d.y;
    return gh - 2.0 * cg;
  }
  static GC_DEV G avg(const G& x, const G& y) {
    G r;
    r.a = scale_(add_(x.a, y.a), T(0.5)); r.b = scale_(add_(x.b, y.b), T(0.5));
    r.c = scale_(add_(x.c, y.c), T(0.5)); r.d = scale_(add_(x.d, y.d), T(0.5));
    return r;
  }
  static GC_DEV T dist2(const G& x, const G& y) {
    return abs2_(sub_(x.a, y.a)) + abs2_(sub_(x.b, y.b)) + abs2_(sub_(x.c, y.c)) + abs2_(sub_(x.d, y.d));
  }
  static GC_DEV T norm2(const G& x) { return abs2_(x.a) + abs2_(x.b) + abs2_(x.c) + abs2_(x.d); }
  static GC_DEV bool finite(const G& x) {
    return isfinite(x.a.x) && isfinite(x.a.y) && isfinite(x.b.x) && isfinite(x.b.y) && isfinite(x.c.x) &&
           isfinite(x.c.y) && isfinite(x.d.x) && isfinite(x.d.y);
  }
  static GC_DEV void write_acc(const T* v, T* jhd, T* jhj, int64_t slot) {
    for (int c = 0; c < 8; ++c) jhd[8 * slot + c] = v[c];
    T* h = jhj + 8 * slot;
    h[0] = v[8]; h[1] = 0; h[2] = v[10]; h[3] = v[11];
    h[4] = v[10]; h[5] = -v[11]; h[6] = v[9]; h[7] = 0;
  }
};

// Moments are stored per interval in tiles of kMomTile baselines as [NM / 4][kMomTile][4] floats:
// a tile is one contiguous block, and the thread that owns a baseline reads its components four at
// a time with 16-byte loads while a warp's loads stay contiguous.  NM is a multiple of 4.
// mom_off counts baseline slots (a multiple of kMomTile per interval).
constexpr int kMomTile = 256;
__host__ __device__ inline int64_t mom_index(int64_t mom_off, int b, int c, int nm) {
  return (mom_off + (b & ~(kMomTile - 1))) * nm + (int64_t)(c >> 2) * (4 * kMomTile) + (b & (kMomTile - 1)) * 4 +
         (c & 3);
}

// ------------------------------------------------------------------------------------------
// Per-baseline moments of an interval (the sample sums with the gains factored out) and the
// per-antenna contributions computed from them; see resident.cu for the algebra.
// ------------------------------------------------------------------------------------------
struct ScalarMom {
  static constexpr int NM = 4;   // Re B, Im B, Q, pad
  static constexpr int AW = 1;   // |g|^2
  static constexpr int BPT = 4;  // baselines per thread in the resident kernel
  using K = ScalarKind<float>;
  static GC_DEV void accum(const float* vis, const float* mod, int64_t r, float* m, float sw) {
    const Cx<float> d = scale_(Vec<float>::ld1(vis + 2 * r), sw), mm = scale_(Vec<float>::ld1(mod + 2 * r), sw);
    m[0] = fma(mm.x, d.x, fma(mm.y, d.y, m[0]));
    m[1] = fma(mm.x, d.y, fma(-mm.y, d.x, m[1]));
    m[2] = fma(mm.x, mm.x, fma(mm.y, mm.y, m[2]));
  }
  static GC_DEV void aux(const K::G& g, float* a) { a[0] = abs2_(g); }
  // p side: c = g_q B, A = |g_q|^2 Q ; q side: c = g_p conj(B), A = |g_p|^2 Q
  static GC_DEV void partials(const float* m, const K::G& gp, const K::G& gq, const float* ap, const float* aq,
                              float* pp, float* pq) {
    const Cx<float> B = cx<float>(m[0], m[1]);
    const Cx<float> cp = mul_(gq, B), cq = mulc_(gp, B);
    pp[0] = cp.x; pp[1] = cp.y; pp[2] = aq[0] * m[2];
    pq[0] = cq.x; pq[1] = cq.y; pq[2] = ap[0] * m[2];
  }
};

struct JonesMom {
  static constexpr int NM = 48;  // P: 4x4 complex row-major (32), R: 4x4 real row-major (16)
  static constexpr int AW = 4;   // G^H G as (a00, a11, Re a01, Im a01)
  static constexpr int BPT = 1;
  using K = JonesKind<float>;
  // P[r][c] += conj(M[i1][j1]) D[i2][j2], r = 2 i1 + i2, c = 2 j1 + j2; R from M (see header).
  static GC_DEV void accum(const float* vis, const float* mod, int64_t r, float* m, float sw) {
    const M2<float> D = scale_m2(Vec<float>::ld4(vis + 8 * r), sw), M = scale_m2(Vec<float>::ld4(mod + 8 * r), sw);
    const Cx<float> Me[4] = {M.a, M.b, M.c, M.d};   // M[i][j] = Me[2 i + j]
    const Cx<float> De[4] = {D.a, D.b, D.c, D.d};
#pragma unroll
    for (int i1 = 0; i1 < 2; ++i1)
#pragma unroll
      for (int i2 = 0; i2 < 2; ++i2)
#pragma unroll
        for (int j1 = 0; j1 < 2; ++j1)
#pragma unroll
          for (int j2 = 0; j2 < 2; ++j2) {
            const int rr = 2 * i1 + i2, cc = 2 * j1 + j2;
            float* e = m + 2 * (rr * 4 + cc);
            cfma2(e[0], e[1], Me[2 * i1 + j1], De[2 * i2 + j2]);
          }
    const Cx<float> u = mulc_(M.a, M.b), v = mulc_(M.c, M.d);
    const Cx<float> w1 = mulc_(M.a, M.c), w2 = mulc_(M.b, M.d), w3 = mulc_(M.a, M.d), w4 = mulc_(M.b, M.c);
    float* R = m + 32;
    R[0] += abs2_(M.a);   R[1] += abs2_(M.b);   R[2] += 2.f * u.x;       R[3] -= 2.f * u.y;
    R[4] += abs2_(M.c);   R[5] += abs2_(M.d);   R[6] += 2.f * v.x;       R[7] -= 2.f * v.y;
    R[8] += w1.x;         R[9] += w2.x;         R[10] += w3.x + w4.x;    R[11] += w4.y - w3.y;
    R[12] += w1.y;        R[13] += w2.y;        R[14] += w3.y + w4.y;    R[15] += w3.x - w4.x;
  }
  static GC_DEV void aux(const K::G& g, float* a) {
    a[0] = abs2_(g.a) + abs2_(g.c);
    a[1] = abs2_(g.b) + abs2_(g.d);
    const Cx<float> o = add_(cmul_(g.a, g.b), cmul_(g.c, g.d));  // (G^H G)_01
    a[2] = o.x;
    a[3] = o.y;
  }
  static GC_DEV void partials(const float* m, const K::G& gp, const K::G& gq, const float* ap, const float* aq,
                              float* pp, float* pq) {
    // p side: vec C = P vec(G_q), vec(G) = [g00, g10, g01, g11]
    const Cx<float> vq[4] = {gq.a, gq.c, gq.b, gq.d};
    const Cx<float> vp[4] = {gp.a, gp.c, gp.b, gp.d};
    Cx<float> c[4], d[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) { c[r] = cx<float>(0.f, 0.f); d[r] = cx<float>(0.f, 0.f); }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const Cx<float> P = cx<float>(m[2 * (r * 4 + k)], m[2 * (r * 4 + k) + 1]);
        fma_(c[r], P, vq[k]);   // (P vec G_q)_r
        cfma_(d[k], P, vp[r]);  // (P^H vec G_p)_k += conj(P[r][k]) vp[r]
      }
    // vec -> row-major [C00, C01, C10, C11] = [v0, v2, v1, v3]
    pp[0] = c[0].x; pp[1] = c[0].y; pp[2] = c[2].x; pp[3] = c[2].y;
    pp[4] = c[1].x; pp[5] = c[1].y; pp[6] = c[3].x; pp[7] = c[3].y;
    pq[0] = d[0].x; pq[1] = d[0].y; pq[2] = d[2].x; pq[3] = d[2].y;
    pq[4] = d[1].x; pq[5] = d[1].y; pq[6] = d[3].x; pq[7] = d[3].y;
    const float* R = m + 32;
    const float w[4] = {1.f, 1.f, 2.f, 2.f};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float hp = 0.f, hq = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        hp = fma(R[i * 4 + j], aq[j], hp);
        hq = fma(R[j * 4 + i] * (w[j] / w[i]), ap[j], hq);  // R' = W^-1 R^T W
      }
      pp[8 + i] = hp;
      pq[8 + i] = hq;
    }
  }
};

}  // namespace gc
