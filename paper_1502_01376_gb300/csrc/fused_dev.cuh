// fused_dev.cuh -- device helpers shared by the fused FP32 2D kernels: complex
// products, twiddles W_R^k as constants, streaming loads and stores,
// release/acquire flags with bounded waits, the kernel arguments, and the job
// record and slot numbers of the round schedule (tm_sched.cuh).
#pragma once
#include "fused_api.cuh"

namespace hyb {

// ------------------------------------------------------------------ complex
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return f2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)); }
__device__ __forceinline__ float2 mulc(float2 a, float2 b) { return f2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y)); }  // a conj(b)

// W_R^k as compile-time constants (forward sign); INV conjugates
template <int R, int K, bool INV>
__device__ __forceinline__ float2 wconst() {
    constexpr double PI = 3.14159265358979323846;
    constexpr int k = ((K % R) + R) % R;
    // cos/sin of 2 pi k / R for the few R used here (exact table of constants)
    constexpr double c = (R == 1 || k == 0) ? 1.0
        : (4 * k == R) ? 0.0 : (2 * k == R) ? -1.0 : (4 * k == 3 * R) ? 0.0
        : (R == 8 && (k == 1 || k == 7)) ? 0.70710678118654752440 : (R == 8) ? -0.70710678118654752440
        : (R == 16) ? ((k == 1 || k == 15) ? 0.92387953251128675613 : (k == 2 || k == 14) ? 0.70710678118654752440
                      : (k == 3 || k == 13) ? 0.38268343236508977173 : (k == 5 || k == 11) ? -0.38268343236508977173
                      : (k == 6 || k == 10) ? -0.70710678118654752440 : -0.92387953251128675613)
        : 0.0;
    constexpr double s = (R == 1 || k == 0 || 2 * k == R) ? 0.0
        : (4 * k == R) ? 1.0 : (4 * k == 3 * R) ? -1.0
        : (R == 8) ? ((k < 4) ? 0.70710678118654752440 : -0.70710678118654752440)
        : (R == 16) ? ((k == 1 || k == 7) ? 0.38268343236508977173 : (k == 2 || k == 6) ? 0.70710678118654752440
                      : (k == 3 || k == 5) ? 0.92387953251128675613 : (k == 9 || k == 15) ? -0.38268343236508977173
                      : (k == 10 || k == 14) ? -0.70710678118654752440 : -0.92387953251128675613)
        : 0.0;
    (void)PI;
    // W_R^k = exp(-2 pi i k / R) = c - i s
    return INV ? f2((float)c, (float)s) : f2((float)c, (float)-s);
}

// W_R^k for R | 16 with k known after unrolling (folds to a constant)
__device__ __forceinline__ float2 wr(int R, int k) {
    const int j = ((k * (16 / R)) % 16 + 16) % 16;      // angle in units of 2 pi / 16
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
    switch (j) {
    case 0: return f2(1.f, 0.f);
    case 1: return f2(c1, -s1);
    case 2: return f2(h, -h);
    case 3: return f2(s1, -c1);
    case 4: return f2(0.f, -1.f);
    case 5: return f2(-s1, -c1);
    case 6: return f2(-h, -h);
    case 7: return f2(-c1, -s1);
    case 8: return f2(-1.f, 0.f);
    case 9: return f2(-c1, s1);
    case 10: return f2(-h, h);
    case 11: return f2(-s1, c1);
    case 12: return f2(0.f, 1.f);
    case 13: return f2(s1, c1);
    case 14: return f2(h, h);
    default: return f2(c1, s1);
    }
}

// ------------------------------------------------------------------ kernel args


__device__ __forceinline__ float2 ldg_stream(const float2* p) {
    float2 v;
    asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
// bounded wait of one thread for flag >= epoch; after `limit` clock cycles (about 2 s
// by default) it sets bit 1 of *err and gives up
constexpr long long kWaitCycles = 4000000000LL;
__device__ __forceinline__ void wait_flag(const int* f, int epoch, int* err, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (ld_acquire(f) < epoch) {
        if (clock64() - t0 > limit) { if (err) atomicOr(err, 2); return; }
        __nanosleep(256);
    }
}
// one row copy by one warp (n a multiple of 4, both rows 16-byte aligned), four float4 in flight a lane
__device__ __forceinline__ void copy_row_warp(const RowCopy& t, int lane) {
    const float4* s4 = reinterpret_cast<const float4*>(t.src);
    float4* d4 = reinterpret_cast<float4*>(t.dst);
    const int n4 = t.n / 4;
    int i = lane;
    for (; i + 96 < n4; i += 128) {
        const float4 a = s4[i], b = s4[i + 32], c = s4[i + 64], d = s4[i + 96];
        d4[i] = a;
        d4[i + 32] = b;
        d4[i + 64] = c;
        d4[i + 96] = d;
    }
    for (; i < n4; i += 32) d4[i] = s4[i];
}
__device__ __forceinline__ void stg_stream(float2* p, float2 v) {
    asm volatile("st.global.L1::no_allocate.v2.f32 [%0], {%1, %2};" :: "l"(p), "f"(v.x), "f"(v.y) : "memory");
}

// job kinds
enum : int { J_IDLE = 0, J_FWD = 1, J_INV = 2 };
// epilogues of forward jobs
enum : int { X_STORE = 0, X_B1, X_B2, X_B3, X_J1, X_J2, X_J3 };

struct Job {
    int kind;
    int epi;          // forward epilogue
    int slot;         // destination slot (forward) or source slot (inverse)
    int row;          // the row p the epilogue refers to
    const float* src; // forward: global source row
    float* dst;       // inverse: global destination row
};

// slot numbers
__device__ __forceinline__ int sE1(int r) { return 0 + (r & 1); }
__device__ __forceinline__ int sE3(int r) { return 2 + (r & 1); }
constexpr int sE2 = 4;
__device__ __forceinline__ int sB1(int r) { return 5 + (r & 1); }
__device__ __forceinline__ int sB3(int r) { return 7 + (r & 1); }
constexpr int sB2 = 9;




}  // namespace hyb
