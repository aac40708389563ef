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

}  // namespace rpa
