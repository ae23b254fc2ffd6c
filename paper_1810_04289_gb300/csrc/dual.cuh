// Forward-mode dual number with one tangent: a + b eps, eps^2 = 0.
// Evaluating an element residual in Dual<T> with one input seeded (tangent 1)
// yields the residual and its exact derivative along that input, i.e. one
// column of the element Jacobian, with the same rounding behaviour as the
// hand-expanded chain rule.
#pragma once
#include <cuda_runtime.h>

template <class T>
struct Dual {
  T v, d;
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(T a) : v(a), d(T(0)) {}
  __host__ __device__ Dual(T a, T b) : v(a), d(b) {}
};

template <class T> __host__ __device__ inline Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> __host__ __device__ inline Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> __host__ __device__ inline Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <class T> __host__ __device__ inline Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> __host__ __device__ inline Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T q = a.v / b.v;
  return Dual<T>(q, (a.d - q * b.d) / b.v);
}
template <class T> __host__ __device__ inline Dual<T> operator+(Dual<T> a, T b) { return Dual<T>(a.v + b, a.d); }
template <class T> __host__ __device__ inline Dual<T> operator+(T a, Dual<T> b) { return Dual<T>(a + b.v, b.d); }
template <class T> __host__ __device__ inline Dual<T> operator-(Dual<T> a, T b) { return Dual<T>(a.v - b, a.d); }
template <class T> __host__ __device__ inline Dual<T> operator-(T a, Dual<T> b) { return Dual<T>(a - b.v, -b.d); }
template <class T> __host__ __device__ inline Dual<T> operator*(Dual<T> a, T b) { return Dual<T>(a.v * b, a.d * b); }
template <class T> __host__ __device__ inline Dual<T> operator*(T a, Dual<T> b) { return Dual<T>(a * b.v, a * b.d); }
template <class T> __host__ __device__ inline Dual<T> operator/(Dual<T> a, T b) { return Dual<T>(a.v / b, a.d / b); }
template <class T> __host__ __device__ inline Dual<T> operator/(T a, Dual<T> b) {
  T q = a / b.v;
  return Dual<T>(q, -q * b.d / b.v);
}
template <class T> __host__ __device__ inline Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a.v += b.v; a.d += b.d; return a; }
template <class T> __host__ __device__ inline Dual<T>& operator-=(Dual<T>& a, Dual<T> b) { a.v -= b.v; a.d -= b.d; return a; }

__device__ inline double dsqrt(double a) { return sqrt(a); }
__device__ inline float dsqrt(float a) { return sqrtf(a); }
template <class T> __device__ inline Dual<T> dsqrt(Dual<T> a) {
  T s = dsqrt(a.v);
  return Dual<T>(s, a.d / (T(2) * s));
}

// value part of a scalar
__device__ inline double val(double a) { return a; }
__device__ inline float val(float a) { return a; }
template <class T> __device__ inline T val(Dual<T> a) { return a.v; }
// tangent part
template <class T> __device__ inline T tan_of(Dual<T> a) { return a.d; }
