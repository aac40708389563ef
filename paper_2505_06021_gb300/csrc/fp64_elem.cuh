// Element type and helpers of the FP64 kernels: one complex128 (interleaved
// re, im) or float64 value, loads, stores and the complex multiply-add in
// four DFMAs.
#pragma once
#include <cuda_runtime.h>

namespace rpa {

template <bool C>
struct Elem;
template <>
struct Elem<true> {
  double re, im;
};
template <>
struct Elem<false> {
  double re;
};

template <bool C>
__device__ __forceinline__ Elem<C> ld_elem(const double* p, long i) {
  Elem<C> e;
  if constexpr (C) {
    double2 v = *reinterpret_cast<const double2*>(p + 2 * i);
    e.re = v.x;
    e.im = v.y;
  } else {
    e.re = p[i];
  }
  return e;
}
template <bool C>
__device__ __forceinline__ Elem<C> zero_elem() {
  Elem<C> e;
  e.re = 0.0;
  if constexpr (C) e.im = 0.0;
  return e;
}
template <bool C>
__device__ __forceinline__ void st_elem(double* p, long i, Elem<C> e) {
  if constexpr (C) {
    *reinterpret_cast<double2*>(p + 2 * i) = make_double2(e.re, e.im);
  } else {
    p[i] = e.re;
  }
}
template <bool C>
__device__ __forceinline__ Elem<C> conj_e(Elem<C> a) {
  if constexpr (C) a.im = -a.im;
  return a;
}
// acc += a * b
template <bool C>
__device__ __forceinline__ void mac(Elem<C>& acc, Elem<C> a, Elem<C> b) {
  if constexpr (C) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
  } else {
    acc.re = fma(a.re, b.re, acc.re);
  }
}

// Float-float form of an element (an unevaluated sum hi + lo of two floats per
// real component, the same size as Elem<C>): the trailing updates of the
// inverse-form log-det run on the FP32 pipe in this arithmetic.
template <bool C>
struct FFE;
template <>
struct FFE<true> {
  float rh, rl, ih, il;
};
template <>
struct FFE<false> {
  float rh, rl;
};
static_assert(sizeof(FFE<true>) == sizeof(Elem<true>) && sizeof(FFE<false>) == sizeof(Elem<false>),
              "float-float and FP64 elements share shared-memory arrays");

template <bool C>
__device__ __forceinline__ FFE<C> to_ff(Elem<C> e) {
  FFE<C> f;
  f.rh = __double2float_rn(e.re);
  f.rl = __double2float_rn(e.re - (double)f.rh);
  if constexpr (C) {
    f.ih = __double2float_rn(e.im);
    f.il = __double2float_rn(e.im - (double)f.ih);
  }
  return f;
}

// Float-float element stored in (and loaded from, through L2) the slot of one
// FP64 element: the two layouts have the same size.
template <bool C>
__device__ __forceinline__ void st_ff(double* p, long i, const FFE<C>& f) {
  if constexpr (C) {
    *reinterpret_cast<float4*>(p + 2 * i) = make_float4(f.rh, f.rl, f.ih, f.il);
  } else {
    *reinterpret_cast<float2*>(p + i) = make_float2(f.rh, f.rl);
  }
}
template <bool C>
__device__ __forceinline__ FFE<C> ld_ff(const double* p, long i) {
  FFE<C> f;
  if constexpr (C) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p + 2 * i));
    f.rh = v.x;
    f.rl = v.y;
    f.ih = v.z;
    f.il = v.w;
  } else {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p + i));
    f.rh = v.x;
    f.rl = v.y;
  }
  return f;
}
template <bool C>
__device__ __forceinline__ FFE<C> conj_ff(FFE<C> f) {
  if constexpr (C) {
    f.ih = -f.ih;
    f.il = -f.il;
  }
  return f;
}

// (h, l) += (ah + al)(bh + bl): the product's rounding error by one fmaf
// (Dekker's TwoProd), the cross terms by two more, the sum's error by Knuth's
// TwoSum; error terms gather in l (renormalised by the caller at the end).
// Explicitly rounded intrinsics keep the compiler from contracting the
// TwoSum into an fma.
__device__ __forceinline__ void ff_mac(float& h, float& l, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = __fadd_rn(h, p);
  const float v = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, v)), __fsub_rn(p, v));
  l = __fadd_rn(l, __fadd_rn(err, e));
  h = s;
}

// acc += a * b in float-float (complex: four real products).
template <bool C>
__device__ __forceinline__ void ff_mac_e(FFE<C>& acc, const FFE<C>& a, const FFE<C>& b) {
  ff_mac(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
  if constexpr (C) {
    ff_mac(acc.rh, acc.rl, -a.ih, -a.il, b.ih, b.il);
    ff_mac(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
    ff_mac(acc.ih, acc.il, a.ih, a.il, b.rh, b.rl);
  }
}

}  // namespace rpa
