// Device helpers shared by the gain-calibration kernels: complex arithmetic on (re, im) pairs,
// 2x2 complex matrices, compensated (Kahan) accumulation and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GC_DEV __device__ __forceinline__

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may start
// before the previous kernel in the stream has finished.  pdl_launch_dependents lets the next
// kernel be scheduled early; pdl_wait blocks until every prerequisite grid has completed and its
// memory is visible (a no-op for a kernel launched without the attribute).
GC_DEV void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
GC_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename T>
struct Cx {
  T x, y;  // re, im
};

template <typename T> GC_DEV Cx<T> cx(T a, T b) { Cx<T> r; r.x = a; r.y = b; return r; }
template <typename T> GC_DEV Cx<T> conj_(Cx<T> a) { return cx<T>(a.x, -a.y); }
template <typename T> GC_DEV Cx<T> add_(Cx<T> a, Cx<T> b) { return cx<T>(a.x + b.x, a.y + b.y); }
template <typename T> GC_DEV Cx<T> sub_(Cx<T> a, Cx<T> b) { return cx<T>(a.x - b.x, a.y - b.y); }
template <typename T> GC_DEV Cx<T> scale_(Cx<T> a, T s) { return cx<T>(a.x * s, a.y * s); }
template <typename T> GC_DEV T abs2_(Cx<T> a) { return fma(a.x, a.x, a.y * a.y); }
// a * b
template <typename T> GC_DEV Cx<T> mul_(Cx<T> a, Cx<T> b) {
  return cx<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> GC_DEV Cx<T> mulc_(Cx<T> a, Cx<T> b) {
  return cx<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
template <typename T> GC_DEV Cx<T> cmul_(Cx<T> a, Cx<T> b) {
  return cx<T>(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// acc += a * b
template <typename T> GC_DEV void fma_(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += a * conj(b)
template <typename T> GC_DEV void fmac_(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
}
// acc += conj(a) * b
template <typename T> GC_DEV void cfma_(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}

// (xr, xi) += a * conj(b)
template <typename T> GC_DEV void fmac2(T& xr, T& xi, Cx<T> a, Cx<T> b) {
  xr = fma(a.x, b.x, fma(a.y, b.y, xr));
  xi = fma(a.y, b.x, fma(-a.x, b.y, xi));
}
// (xr, xi) += conj(a) * b
template <typename T> GC_DEV void cfma2(T& xr, T& xi, Cx<T> a, Cx<T> b) {
  xr = fma(a.x, b.x, fma(a.y, b.y, xr));
  xi = fma(a.x, b.y, fma(-a.y, b.x, xi));
}

// 2x2 complex matrix [[a, b], [c, d]] (row-major storage order a, b, c, d).
template <typename T>
struct M2 {
  Cx<T> a, b, c, d;
};

template <typename T> GC_DEV M2<T> mm_(const M2<T>& X, const M2<T>& Y) {  // X Y
  M2<T> r;
  r.a = mul_(X.a, Y.a); fma_(r.a, X.b, Y.c);
  r.b = mul_(X.a, Y.b); fma_(r.b, X.b, Y.d);
  r.c = mul_(X.c, Y.a); fma_(r.c, X.d, Y.c);
  r.d = mul_(X.c, Y.b); fma_(r.d, X.d, Y.d);
  return r;
}
template <typename T> GC_DEV M2<T> mmh_(const M2<T>& X, const M2<T>& Y) {  // X Y^H
  M2<T> r;
  r.a = mulc_(X.a, Y.a); fmac_(r.a, X.b, Y.b);
  r.b = mulc_(X.a, Y.c); fmac_(r.b, X.b, Y.d);
  r.c = mulc_(X.c, Y.a); fmac_(r.c, X.d, Y.b);
  r.d = mulc_(X.c, Y.c); fmac_(r.d, X.d, Y.d);
  return r;
}

// Vector loads of one row.  float: complex64 (8 bytes); a 2x2 row is 32 bytes = 2 x float4.
template <typename T> struct Vec;
template <> struct Vec<float> {
  static GC_DEV Cx<float> ld1(const float* p) {
    float2 v = __ldcs(reinterpret_cast<const float2*>(p));
    return cx<float>(v.x, v.y);
  }
  static GC_DEV M2<float> ld4(const float* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    float4 u = __ldcs(q), v = __ldcs(q + 1);
    M2<float> m;
    m.a = cx<float>(u.x, u.y); m.b = cx<float>(u.z, u.w);
    m.c = cx<float>(v.x, v.y); m.d = cx<float>(v.z, v.w);
    return m;
  }
};
template <> struct Vec<double> {
  static GC_DEV Cx<double> ld1(const double* p) {
    double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    return cx<double>(v.x, v.y);
  }
  static GC_DEV M2<double> ld4(const double* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 u0 = __ldcs(q), u1 = __ldcs(q + 1), u2 = __ldcs(q + 2), u3 = __ldcs(q + 3);
    M2<double> m;
    m.a = cx<double>(u0.x, u0.y); m.b = cx<double>(u1.x, u1.y);
    m.c = cx<double>(u2.x, u2.y); m.d = cx<double>(u3.x, u3.y);
    return m;
  }
};

// Compensated (Kahan) addition of v into (s, c); the value is s - c.
template <typename T> GC_DEV void kahan_add(T& s, T& c, T v) {
  T y = v - c;
  T t = s + y;
  c = (t - s) - y;
  s = t;
}

// Deterministic block-wide sum (fixed shuffle tree, fixed warp order).  `red` holds >= 32 T.
template <typename T> GC_DEV T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T r = 0;
  if (warp == 0) {
    r = lane < nw ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) red[0] = r;
  }
  __syncthreads();
  r = red[0];
  __syncthreads();
  return r;
}

GC_DEV int block_or(int v, int* red) {
  v = __any_sync(0xffffffffu, v) ? 1 : 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int r = 0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int w = 0; w < nw; ++w) r |= red[w];
  __syncthreads();
  return r;
}

// Float-float ("double-float") arithmetic on the FP32 pipe: an unevaluated sum hi + lo with
// |lo| <= ulp(hi) / 2.  Knuth's TwoSum gives a sum's rounding error exactly; an FMA gives a
// product's (the TwoProduct of Ogita, Rump and Oishi).  GB300 runs FP32 many times faster than
// FP64, so sums that want more than FP32 precision are kept in these pairs instead of in doubles.
struct FF {
  float hi, lo;
};
// (the _rn intrinsics are never contracted into FMAs, which would break the exact error terms)
GC_DEV FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
GC_DEV FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  const float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  const float hi = __fadd_rn(s.hi, lo);  // renormalise (fast TwoSum, |s.hi| >= |lo|)
  return FF{hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}
// x - a * b, with the product's rounding error carried into lo
GC_DEV FF ff_sub_prod(FF x, float a, float b) {
  const float p = __fmul_rn(a, b), e = __fmaf_rn(a, b, -p);
  const FF s = ff_two_sum(x.hi, -p);
  const float lo = __fadd_rn(s.lo, __fsub_rn(x.lo, e));
  const float hi = __fadd_rn(s.hi, lo);
  return FF{hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}

GC_DEV FF ff_add_f(FF x, float v) { return ff_add(x, FF{v, 0.f}); }
GC_DEV double ff_value(FF x) { return (double)x.hi + (double)x.lo; }

// End-of-update reduction over the block with the two sums in float-float: every thread gets the
// block totals of d2 and n2 (warp butterflies, then the warps in order) and the OR of the two
// flags; two barriers.  Only the first n_live threads may hold nonzero values or set flags: the
// warps past them skip the butterfly and are left out of the totals.  `red` holds >= 160 floats.
GC_DEV void block_reduce_step_ff(FF& d2, FF& n2, int& f1, int& f2, float* red, int n_live) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (min(n_live, (int)blockDim.x) + 31) >> 5;
  int fl = (f1 ? 1 : 0) | (f2 ? 2 : 0);
  if (warp < nw) {  // warp-uniform
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      d2 = ff_add(d2, FF{__shfl_xor_sync(0xffffffffu, d2.hi, o), __shfl_xor_sync(0xffffffffu, d2.lo, o)});
      n2 = ff_add(n2, FF{__shfl_xor_sync(0xffffffffu, n2.hi, o), __shfl_xor_sync(0xffffffffu, n2.lo, o)});
      fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    }
  }
  if (lane == 0 && warp < nw) {
    red[warp] = d2.hi;
    red[32 + warp] = d2.lo;
    red[64 + warp] = n2.hi;
    red[96 + warp] = n2.lo;
    red[128 + warp] = __int_as_float(fl);
  }
  __syncthreads();
  FF a{0.f, 0.f}, b{0.f, 0.f};
  int f = 0;
  for (int w = 0; w < nw; ++w) {
    a = ff_add(a, FF{red[w], red[32 + w]});
    b = ff_add(b, FF{red[64 + w], red[96 + w]});
    f |= __float_as_int(red[128 + w]);
  }
  __syncthreads();
  d2 = a;
  n2 = b;
  f1 = f & 1;
  f2 = (f >> 1) & 1;
}


// Fixed-order reduction of one tile's per-slot partial sums into per-antenna sums.  `off`/`ent`
// give, per antenna, the list of partial-sum slots (float offsets into `part`).  Each list is cut
// into CH equal chunks summed in parallel (long lists -- e.g. an antenna's p side over a run of
// consecutive baselines -- would otherwise serialise the tile), then the chunk sums are added in
// chunk order and compensated into (acc, cmp).  `ps` holds nat * NC * CH floats.
template <int NC, int CH>
GC_DEV void tile_reduce(const float* part, const int* off, const int* ent, int nat, float* acc, float* cmp,
                        float* ps) {
  for (int x = threadIdx.x; x < nat * NC * CH; x += blockDim.x) {
    const int ch = x % CH, r = x / CH, an = r / NC, c = r - an * NC;
    const int e0 = __ldg(off + an), len = __ldg(off + an + 1) - e0;
    const int b0 = e0 + (len * ch) / CH, b1 = e0 + (len * (ch + 1)) / CH;
    float s0 = 0.f, s1 = 0.f;
    int e = b0;
    for (; e + 1 < b1; e += 2) {
      s0 += part[__ldg(ent + e) + c];
      s1 += part[__ldg(ent + e + 1) + c];
    }
    if (e < b1) s0 += part[__ldg(ent + e) + c];
    ps[x] = s0 + s1;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nat * NC; x += blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int ch = 0; ch < CH; ++ch) s += ps[x * CH + ch];
    kahan_add(acc[x], cmp[x], s);
  }
}
