// goc_vec.cuh -- one collision source for one node (float) or two nodes at
// once (float2 on the packed f32x2 add/mul/fma of sm_100-family GPUs, one
// instruction for both lanes).  Every operation is rounded to nearest, lane by
// lane, so a float2 lane computes exactly what the float form computes when the
// float form is written with the same explicit fma's.
#pragma once

#include <cuda_runtime.h>

namespace goc {

template <class V> struct Lanes;
template <> struct Lanes<float> { static constexpr int R = 1; };
template <> struct Lanes<float2> { static constexpr int R = 2; };

template <class V> __device__ __forceinline__ V bc(float s);
template <> __device__ __forceinline__ float bc<float>(float s) { return s; }
template <> __device__ __forceinline__ float2 bc<float2>(float s) { return make_float2(s, s); }

// value of lane k / a V from R lane values
__device__ __forceinline__ float lane(float v, int) { return v; }
__device__ __forceinline__ float lane(float2 v, int k) { return k ? v.y : v.x; }
template <class V> __device__ __forceinline__ V pack(const float *a);
template <> __device__ __forceinline__ float pack<float>(const float *a) { return a[0]; }
template <> __device__ __forceinline__ float2 pack<float2>(const float *a) { return make_float2(a[0], a[1]); }

__device__ __forceinline__ float fmav(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 fmav(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmav(float a, float2 b, float2 c) { return __ffma2_rn(make_float2(a, a), b, c); }
__device__ __forceinline__ float2 fmav(float2 a, float b, float2 c) { return __ffma2_rn(a, make_float2(b, b), c); }
__device__ __forceinline__ float2 fmav(float2 a, float2 b, float c) { return __ffma2_rn(a, b, make_float2(c, c)); }
__device__ __forceinline__ float2 fmav(float a, float2 b, float c) {
    return __ffma2_rn(make_float2(a, a), b, make_float2(c, c));
}
__device__ __forceinline__ float2 fmav(float2 a, float b, float c) {
    return __ffma2_rn(a, make_float2(b, b), make_float2(c, c));
}

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b as b * (-1) + a: the product is exact, so this is the rounded difference
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 operator-(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }
__device__ __forceinline__ float2 operator+(float2 a, float s) { return __fadd2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 operator+(float s, float2 a) { return __fadd2_rn(make_float2(s, s), a); }
__device__ __forceinline__ float2 operator-(float2 a, float s) { return __fadd2_rn(a, make_float2(-s, -s)); }
__device__ __forceinline__ float2 operator-(float s, float2 a) {
    return __ffma2_rn(a, make_float2(-1.f, -1.f), make_float2(s, s));
}
__device__ __forceinline__ float2 operator*(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return __fmul2_rn(make_float2(s, s), a); }

__device__ __forceinline__ float rcpv(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float2 rcpv(float2 x) { return make_float2(__frcp_rn(x.x), __frcp_rn(x.y)); }

}  // namespace goc
