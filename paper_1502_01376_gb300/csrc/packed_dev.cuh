// packed_dev.cuh -- packed FP32 pair arithmetic (add/sub/mul/fma.rn.f32x2) and the
// 4- and 8-point DFTs built on it, shared by the fused kernel and the row FFTs.
#pragma once
#include <cuda_runtime.h>

namespace hyb {

__device__ __forceinline__ float2 pf2(float a, float b) { return make_float2(a, b); }

// ------------------------------------------------------------------ packed FP32 pairs (f32x2): one instruction
// for the two components of a complex add, subtract or scale
__device__ __forceinline__ unsigned long long pk(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
// a * b + c per component
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(r);
}

// 4-point DFT (natural order) with packed adds: the rotation by -i (+i for
// the inverse) of the odd difference is folded into four scalar adds
template <bool INV>
__device__ __forceinline__ void dft4x(float2& x0, float2& x1, float2& x2, float2& x3) {
    const float2 A = vadd(x0, x2), B = vsub(x0, x2), C = vadd(x1, x3), Y = vsub(x1, x3);
    x0 = vadd(A, C);
    x2 = vsub(A, C);
    if (!INV) { x1 = pf2(B.x + Y.y, B.y - Y.x); x3 = pf2(B.x - Y.y, B.y + Y.x); }
    else { x1 = pf2(B.x - Y.y, B.y + Y.x); x3 = pf2(B.x + Y.y, B.y - Y.x); }
}
// 8-point DFT (natural order): two 4-point DFTs, twiddles W_8^k, radix-2 combine
template <bool INV>
__device__ __forceinline__ void dft8x(float2 (&x)[8]) {
    float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4x<INV>(e0, e1, e2, e3);
    dft4x<INV>(o0, o1, o2, o3);
    const float h = 0.70710678118654752440f;
    // o1 W_8^1 and o3 W_8^3 (conjugated for the inverse)
    if (!INV) {
        o1 = vmul(pf2(o1.x + o1.y, o1.y - o1.x), pf2(h, h));
        o3 = vmul(pf2(o3.y - o3.x, o3.x + o3.y), pf2(h, -h));
    } else {
        o1 = vmul(pf2(o1.x - o1.y, o1.x + o1.y), pf2(h, h));
        o3 = vmul(pf2(o3.x + o3.y, o3.x - o3.y), pf2(-h, h));
    }
    x[0] = vadd(e0, o0); x[4] = vsub(e0, o0);
    x[1] = vadd(e1, o1); x[5] = vsub(e1, o1);
    x[3] = vadd(e3, o3); x[7] = vsub(e3, o3);
    // o2 times -i (forward) or +i (inverse)
    if (!INV) { x[2] = pf2(e2.x + o2.y, e2.y - o2.x); x[6] = pf2(e2.x - o2.y, e2.y + o2.x); }
    else { x[2] = pf2(e2.x - o2.y, e2.y + o2.x); x[6] = pf2(e2.x + o2.y, e2.y - o2.x); }
}


}  // namespace hyb
