// Packed FP32 pairs.  Compute capability 10.x executes add, sub, mul and fma
// on a pair of FP32 values (PTX .f32x2) as one instruction; each half is
// rounded exactly as the scalar operation would be.  A pair lives in one
// 64-bit register pair, the low half first.  min, max and negation have no
// packed form.
#pragma once

namespace f32x2 {

typedef unsigned long long f2p;          // two packed floats, low half first
__device__ __forceinline__ f2p pk2(float a, float b) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f2p r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p add2_rd(f2p a, f2p b) {
    f2p d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p splat2(float a) { return pk2(a, a); }

}  // namespace f32x2
