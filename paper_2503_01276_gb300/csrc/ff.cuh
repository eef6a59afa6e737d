// Float-float ("double-word") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits (relative rounding ~ 2^-47).
//
// On this GPU an FP64 FMA runs at about 1/64 of the FP32 rate and an FP64 -> FP32
// conversion at about twice the FP64 FMA rate, so FP64-bound work on vectors kept in this
// format (two float planes of the same size as one FP64 vector) runs on the FP32 pipes.
//
// Building blocks (error-free transformations):
//   two_sum       Knuth's branch-free exact sum: s + e == a + b exactly.
//   fast_two_sum  Dekker's exact sum for |a| >= |b| (or a == 0).
//   two_prod      exact product with one FMA: p + e == a * b exactly.
// Word operations follow the double-word algorithms of Joldes, Muller and Popescu
// ("Tight and rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 2017), u = 2^-24: the sum is their "sloppy" double-word sum (one two_sum on the
// high words; absolute error about 2u^2 (|a| + |b|), i.e. bounded like an FP64 sum's by the
// operands' size rather than the result's, which is all the stencils, interpolations and
// reductions here need), the products use one or two FMAs (relative error <= 5u^2 / 4u^2).
//
// Storage: a vector of nv entries occupies the space of nv doubles as a hi plane [nv] followed
// by a lo plane [nv].
#pragma once

#include <cuda_runtime.h>

namespace mch {

struct ff {
  float h, l;
};

// The _rn intrinsics are never contracted into FMAs, which would break exactness.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_from(double d) {
  const float h = (float)d;
  return ff{h, (float)(d - (double)h)};
}
__device__ __forceinline__ double ff_to(ff a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ ff ff_of(float f) { return ff{f, 0.f}; }

__device__ __forceinline__ ff operator+(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  fast_two_sum(s, e, s, e);
  return ff{s, e};
}
__device__ __forceinline__ ff operator-(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  float s, t;
  fast_two_sum(p, e, s, t);
  return ff{s, t};
}
__device__ __forceinline__ ff operator*(ff a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return ff{s, t};
}
__device__ __forceinline__ ff operator*(float b, ff a) { return a * b; }
__device__ __forceinline__ ff &operator+=(ff &a, ff b) { return a = a + b; }
__device__ __forceinline__ ff &operator-=(ff &a, ff b) { return a = a - b; }

// acc += p
__device__ __forceinline__ void ff_acc(ff &acc, ff p) { acc = acc + p; }

// Exact scaling by a power of two.
__device__ __forceinline__ ff ff_scale2(ff a, float pow2) { return ff{a.h * pow2, a.l * pow2}; }

// Sum of products of double-words in the manner of Ogita, Rump and Oishi's Dot2 ("Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005): the high words' products are split
// exactly (two_prod) and summed with two_sum into s; every rounding error of those steps and
// the cross terms a.h b.l + a.l b.h (themselves ~u of the product) go into one FP32 word e.
// About 11 FP32 instructions per term instead of ~18 for a double-word product and sum, with
// an error of the same kind (~n u^2 times the sum of the terms' magnitudes).
struct ffdot {
  float s, e;
};
__device__ __forceinline__ void dot_add(ffdot &d, ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  const float pe = __fmaf_rn(a.h, b.h, -p);
  float s, t;
  two_sum(d.s, p, s, t);
  d.s = s;
  d.e = __fadd_rn(d.e, __fadd_rn(t, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, pe))));
}
__device__ __forceinline__ void dot_add(ffdot &d, ff a) {
  float s, t;
  two_sum(d.s, a.h, s, t);
  d.s = s;
  d.e = __fadd_rn(d.e, __fadd_rn(t, a.l));
}
__device__ __forceinline__ ff dot_get(ffdot d) {
  float s, e;
  two_sum(d.s, d.e, s, e);
  return ff{s, e};
}

// plane access: vector v (index of a whole vector) of a batch with stride nv entries
__device__ __forceinline__ ff ff_load(const double *base, size_t v, int nv, int k) {
  const float *p = reinterpret_cast<const float *>(base) + v * 2 * (size_t)nv;
  return ff{p[k], p[nv + k]};
}
__device__ __forceinline__ void ff_store(double *base, size_t v, int nv, int k, ff x) {
  float *p = reinterpret_cast<float *>(base) + v * 2 * (size_t)nv;
  p[k] = x.h;
  p[nv + k] = x.l;
}

// Storage traits of level-1-grid vectors: FP64 or float-float planes, with the loads,
// stores, conversions and the two reduction helpers the kernels need.
struct F64S {
  using V = double;
  using P = double *;
  // base of vector v, then entry k of it with 32-bit offsets
  __device__ static P vec(const double *b, size_t v, int nv) { return const_cast<P>(b) + v * nv; }
  __device__ static V ldv(P p, int, int k) { return p[k]; }
  __device__ static void stv(P p, int, int k, V x) { p[k] = x; }
  __device__ static V ld(const double *b, size_t v, int nv, int k) { return b[v * nv + k]; }
  __device__ static void st(double *b, size_t v, int nv, int k, V x) { b[v * nv + k] = x; }
  __device__ static V from(double d) { return d; }
  __device__ static V fromf(float f) { return (double)f; }
  __device__ static double to(V x) { return x; }
  __device__ static V zero() { return 0.0; }
  __device__ static V shfl_xor(V v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  // sums of products (Dot2 accumulator in float-float storage)
  using D = double;
  __device__ static D dzero() { return 0.0; }
  __device__ static void dadd(D &d, V a, V b) { d += a * b; }
  __device__ static void dadd(D &d, V a) { d += a; }
  __device__ static V dget(D d) { return d; }
  __device__ static V scale2(V a, float p2) { return a * (double)p2; }
};

struct FFS {
  using V = ff;
  using P = float *;
  __device__ static P vec(const double *b, size_t v, int nv) {
    return const_cast<float *>(reinterpret_cast<const float *>(b)) + v * 2 * (size_t)nv;
  }
  __device__ static V ldv(P p, int nv, int k) { return ff{p[k], p[nv + k]}; }
  __device__ static void stv(P p, int nv, int k, V x) {
    p[k] = x.h;
    p[nv + k] = x.l;
  }
  __device__ static V ld(const double *b, size_t v, int nv, int k) { return ff_load(b, v, nv, k); }
  __device__ static void st(double *b, size_t v, int nv, int k, V x) { ff_store(b, v, nv, k, x); }
  __device__ static V from(double d) { return ff_from(d); }
  __device__ static V fromf(float f) { return ff{f, 0.f}; }
  __device__ static double to(V x) { return ff_to(x); }
  __device__ static V zero() { return ff{0.f, 0.f}; }
  __device__ static V shfl_xor(V v, int o) {
    return ff{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
  }
  using D = ffdot;
  __device__ static D dzero() { return ffdot{0.f, 0.f}; }
  __device__ static void dadd(D &d, V a, V b) { dot_add(d, a, b); }
  __device__ static void dadd(D &d, V a) { dot_add(d, a); }
  __device__ static V dget(D d) { return dot_get(d); }
  __device__ static V scale2(V a, float p2) { return ff_scale2(a, p2); }
};

}  // namespace mch
