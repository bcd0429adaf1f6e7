// Arithmetic on pairs of opposite populations (2p+1, 2p+2).
//
// Many DUGKS operations apply the same coefficient pattern to both members of
// a pair.  For FP32 the pair is a float2 and each operation is one packed
// FP32x2 instruction (sm_100 and later); FP64 falls back to two scalar
// operations.  Every packed operation rounds each lane exactly like the
// scalar operation it replaces.
#pragma once

#include <cuda_runtime.h>

#ifndef KIN_PACK_F32X2
#define KIN_PACK_F32X2 1
#endif

namespace kin {

template <typename C>
struct PairOf;
template <>
struct PairOf<float> {
    using T = float2;
};
template <>
struct PairOf<double> {
    using T = double2;
};
template <typename C>
using Pr = typename PairOf<C>::T;

__host__ __device__ __forceinline__ float2 pmk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 pmk(double a, double b) { return make_double2(a, b); }

// ---- FP32
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
#if KIN_PACK_F32X2
    return __fadd2_rn(a, b);
#else
    return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
#endif
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
#if KIN_PACK_F32X2
    return __fmul2_rn(a, b);
#else
    return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
#endif
}
// a * b + c, one rounding per lane
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
#if KIN_PACK_F32X2
    return __ffma2_rn(a, b, c);
#else
    return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
#endif
}
// a - b, written as b * (-1) + a so that it is a single packed instruction
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
#if KIN_PACK_F32X2
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
#else
    return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
#endif
}
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }

// ---- FP64 (scalar lanes)
__device__ __forceinline__ double2 padd(double2 a, double2 b) {
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 pmul(double2 a, double2 b) {
    return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) {
    return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}
__device__ __forceinline__ double2 pneg(double2 a) { return make_double2(-a.x, -a.y); }

// acc + SG * v for a compile-time sign SG = +1 or -1
template <int SG, typename T>
__device__ __forceinline__ T padd_sg(T acc, T v) {
    if constexpr (SG > 0) return padd(acc, v);
    else return psub(acc, v);
}

}  // namespace kin
