// Two FP32 values in one 64-bit register pair, with the packed sm_100-family
// instructions add/sub/mul/fma.rn.f32x2: one instruction evaluates the same
// operation for two independent elements, so the element routine, written once
// for a scalar type T, evaluates two elements for the issue cost of one.  Each
// component is rounded exactly as the scalar FP32 operation would be.
#pragma once

namespace jfnk {

struct pf2 {
    unsigned long long v;
    pf2() = default;
    // both components equal to c (rounded to FP32)
    __device__ __forceinline__ explicit pf2(double c) {
        const float f = (float)c;
        asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(f));
    }
};

__device__ __forceinline__ pf2 pf2_pack(float lo, float hi) {
    pf2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void pf2_unpack(pf2 a, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
// the pair stored at p (8-byte aligned): lo = p[0], hi = p[1]
__device__ __forceinline__ pf2 pf2_load(const float* p) {
    pf2 r;
    r.v = *reinterpret_cast<const unsigned long long*>(p);
    return r;
}
__device__ __forceinline__ void pf2_store(float* p, pf2 a) { *reinterpret_cast<unsigned long long*>(p) = a.v; }

__device__ __forceinline__ pf2 operator+(pf2 a, pf2 b) {
    pf2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ pf2 operator-(pf2 a, pf2 b) {
    pf2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ pf2 operator*(pf2 a, pf2 b) {
    pf2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ pf2 operator-(pf2 a) { return pf2(0.0) - a; }
// a b + c with one rounding per component
__device__ __forceinline__ pf2 madd(pf2 a, pf2 b, pf2 c) {
    pf2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

}  // namespace jfnk
