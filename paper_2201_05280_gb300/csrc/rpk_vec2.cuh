// Two FP32 lanes -- the same quantity at two lattice points -- in one value.
// Every arithmetic operator is one packed FP32x2 instruction of the sm_100
// family (add / mul / fma .f32x2, round to nearest, never contracted), so
// that a kernel written once over a value type V runs for V = float (one
// point) and V = F2 (two points), the packed form issuing half the arithmetic
// instructions per point. The two forms agree to FP32 rounding, not bit for
// bit: on random inputs about a fifth of the moments differ in the last bits
// between the two instantiations, with or without contraction of the scalar
// code.
#pragma once

#include <cuda_runtime.h>

namespace rpk {

struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ explicit F2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit F2(float2 a) : v(a) {}
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
// a - b = fma(b, -1, a): exact product, one rounding, as the scalar subtraction
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  return F2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
// mixed forms: the scalar is the same at both points
__device__ __forceinline__ F2 operator+(F2 a, float b) { return a + F2(b); }
__device__ __forceinline__ F2 operator+(float a, F2 b) { return F2(a) + b; }
__device__ __forceinline__ F2 operator-(F2 a, float b) { return a - F2(b); }
__device__ __forceinline__ F2 operator-(float a, F2 b) { return F2(a) - b; }
__device__ __forceinline__ F2 operator*(F2 a, float b) { return a * F2(b); }
__device__ __forceinline__ F2 operator*(float a, F2 b) { return F2(a) * b; }
__device__ __forceinline__ F2 operator/(float a, F2 b) { return F2(a / b.v.x, a / b.v.y); }
__device__ __forceinline__ F2 operator/(F2 a, float b) { return F2(a.v.x / b, a.v.y / b); }

// a * b + c with a single rounding
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 fmad(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 fmad(float a, F2 b, F2 c) { return fmad(F2(a), b, c); }
__device__ __forceinline__ F2 fmad(F2 a, float b, F2 c) { return fmad(a, F2(b), c); }

// Scalar type of a value type: the type of the per-launch constants.
template <typename V>
struct ScalarOf {
  using type = V;
};
template <>
struct ScalarOf<F2> {
  using type = float;
};
template <typename V>
using scalar_t = typename ScalarOf<V>::type;

// A value with every lane equal to the scalar a.
template <typename V>
__device__ __forceinline__ V splat(scalar_t<V> a) {
  return V(a);
}

}  // namespace rpk
