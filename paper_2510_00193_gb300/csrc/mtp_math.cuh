// Scalar helpers shared by the generated MTP level code and the kernels.
#pragma once
#include <cmath>
#include <type_traits>

#ifndef __CUDACC__
#define __device__
#define __host__
#define __forceinline__ inline
// host compilation of the generated code (tests): one thread stands for the warp
inline void __syncwarp(unsigned = 0xffffffffu) {}
#endif

namespace mtp {

// Forward-mode dual number: value and tangent along one direction.  Used to
// differentiate the whole force evaluation once more (double backward).
template <class S>
struct Dual {
  S v, t;
  __host__ __device__ Dual() : v(0), t(0) {}
  __host__ __device__ Dual(S a) : v(a), t(0) {}
  __host__ __device__ Dual(S a, S b) : v(a), t(b) {}
};

template <class S> __host__ __device__ __forceinline__ Dual<S> operator+(Dual<S> a, Dual<S> b) { return {a.v + b.v, a.t + b.t}; }
template <class S> __host__ __device__ __forceinline__ Dual<S> operator-(Dual<S> a, Dual<S> b) { return {a.v - b.v, a.t - b.t}; }
template <class S> __host__ __device__ __forceinline__ Dual<S> operator-(Dual<S> a) { return {-a.v, -a.t}; }
template <class S> __host__ __device__ __forceinline__ Dual<S> operator*(Dual<S> a, Dual<S> b) { return {a.v * b.v, a.v * b.t + a.t * b.v}; }
template <class S> __host__ __device__ __forceinline__ Dual<S>& operator+=(Dual<S>& a, Dual<S> b) { a.v += b.v; a.t += b.t; return a; }

template <class R> struct ScalarOf { using T = R; };
template <class S> struct ScalarOf<Dual<S>> { using T = S; };

__host__ __device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
template <class S>
__host__ __device__ __forceinline__ Dual<S> fmadd(Dual<S> a, Dual<S> b, Dual<S> c) {
  return {fmadd(a.v, b.v, c.v), fmadd(a.v, b.t, fmadd(a.t, b.v, c.t))};
}

// Optimisation barrier: afterwards the compiler must treat x as an unknown
// value, so expressions of it are formed anew rather than merged with the same
// expressions of the value before (the generated contraction uses this to
// recompute DAG nodes in its reverse pass instead of keeping them live).
__host__ __device__ __forceinline__ void opaque(float& x) {
#ifdef __CUDA_ARCH__
  asm volatile("" : "+f"(x));
#else
  (void)x;
#endif
}
__host__ __device__ __forceinline__ void opaque(double& x) {
#ifdef __CUDA_ARCH__
  asm volatile("" : "+d"(x));
#else
  (void)x;
#endif
}
template <class S> __host__ __device__ __forceinline__ void opaque(Dual<S>& x) {
  opaque(x.v);
  opaque(x.t);
}

// Where the contraction puts basis value a: an array, or a sink object
// called as sink(a, value) (which may reduce it at once).
template <class R> __host__ __device__ __forceinline__ void store_basis(R* B, int a, R v) { B[a] = v; }
template <class Sink, class R> __host__ __device__ __forceinline__ void store_basis(const Sink& B, int a, R v) {
  B(a, v);
}

template <class R> __host__ __device__ __forceinline__ typename ScalarOf<R>::T value_of(R a) { return a; }
template <class S> __host__ __device__ __forceinline__ S value_of(Dual<S> a) { return a.v; }

}  // namespace mtp
