// fused_dev.cuh -- device helpers shared by the fused FP32 2D kernels:
// complex arithmetic, small DFTs with constant twiddles, streaming loads and
// stores, release/acquire flags with bounded waits, and the round schedule
// (which row, slot and epilogue each thread group handles in each round).
#pragma once
#include "fused_api.cuh"

namespace hyb {

// ------------------------------------------------------------------ complex
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return f2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)); }
__device__ __forceinline__ float2 mulc(float2 a, float2 b) { return f2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y)); }  // a conj(b)
__device__ __forceinline__ float2 scl(float2 a, float s) { return f2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 conjf2(float2 a) { return f2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 rot(float2 a) { return INV ? f2(-a.y, a.x) : f2(a.y, -a.x); }

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

// ------------------------------------------------------------------ small DFTs (natural order in/out)
template <bool INV> __device__ __forceinline__ void dft2(float2& a, float2& b) { float2 t = a; a = add(t, b); b = sub(t, b); }

template <bool INV> __device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    float2 a = add(x0, x2), b = sub(x0, x2), c = add(x1, x3), d = rot<INV>(sub(x1, x3));
    x0 = add(a, c); x2 = sub(a, c); x1 = add(b, d); x3 = sub(b, d);
}

template <int R, bool INV> struct Dft;
template <bool INV> struct Dft<1, INV> { template <typename A> __device__ static void run(A&) {} };
template <bool INV> struct Dft<2, INV> { template <typename A> __device__ static void run(A& x) { dft2<INV>(x[0], x[1]); } };
template <bool INV> struct Dft<4, INV> { template <typename A> __device__ static void run(A& x) { dft4<INV>(x[0], x[1], x[2], x[3]); } };
template <bool INV> struct Dft<8, INV> {
    template <typename A> __device__ static void run(A& x) {
        // n = 2 n1 + n2, k = k1 + 4 k2
        float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
        float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
        dft4<INV>(e0, e1, e2, e3);
        dft4<INV>(o0, o1, o2, o3);
        o1 = mul(o1, wconst<8, 1, INV>());
        o2 = rot<INV>(o2);
        o3 = mul(o3, wconst<8, 3, INV>());
        x[0] = add(e0, o0); x[4] = sub(e0, o0);
        x[1] = add(e1, o1); x[5] = sub(e1, o1);
        x[2] = add(e2, o2); x[6] = sub(e2, o2);
        x[3] = add(e3, o3); x[7] = sub(e3, o3);
    }
};
template <bool INV> struct Dft<16, INV> {
    template <typename A> __device__ static void run(A& x) {
        // n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W16^{n2 k1}, DFT4 over n2
        float2 y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; n2++) {
            y[n2][0] = x[n2]; y[n2][1] = x[4 + n2]; y[n2][2] = x[8 + n2]; y[n2][3] = x[12 + n2];
            dft4<INV>(y[n2][0], y[n2][1], y[n2][2], y[n2][3]);
        }
        y[1][1] = mul(y[1][1], wconst<16, 1, INV>());
        y[1][2] = mul(y[1][2], wconst<16, 2, INV>());
        y[1][3] = mul(y[1][3], wconst<16, 3, INV>());
        y[2][1] = mul(y[2][1], wconst<16, 2, INV>());
        y[2][2] = rot<INV>(y[2][2]);
        y[2][3] = mul(y[2][3], wconst<16, 6, INV>());
        y[3][1] = mul(y[3][1], wconst<16, 3, INV>());
        y[3][2] = mul(y[3][2], wconst<16, 6, INV>());
        y[3][3] = mul(y[3][3], wconst<16, 9, INV>());
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++) {
            float2 a = y[0][k1], b = y[1][k1], c = y[2][k1], d = y[3][k1];
            dft4<INV>(a, b, c, d);
            x[k1] = a; x[k1 + 4] = b; x[k1 + 8] = c; x[k1 + 12] = d;
        }
    }
};

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
constexpr int kSlots = 10;


// job of group g in round index ri of a strip [p0, p1)
__device__ __forceinline__ Job job_of(const FusedInst& a, int N, int strip, int p0, int p1, int ri, int g) {
    Job j{J_IDLE, X_STORE, 0, 0, nullptr, nullptr};
    const float* halo = a.halo + (size_t)strip * 7 * N;
    const int h = p0 - 1;
    if (ri < 3) {
        if (ri == 0) {
            j.kind = J_FWD; j.epi = X_STORE;
            if (g == 0) { j.src = a.E[0] + (size_t)p0 * N; j.slot = sE1(p0); }
            else if (g == 1) { j.src = a.E[2] + (size_t)p0 * N; j.slot = sE3(p0); }
            else { j.src = halo + 1 * N; j.slot = sE2; }
        } else if (ri == 1) {
            if (g == 0) { j.kind = J_FWD; j.epi = X_STORE; j.src = halo + 0 * N; j.slot = sE1(h); }
            else if (g == 1) { j.kind = J_FWD; j.epi = X_STORE; j.src = halo + 2 * N; j.slot = sE3(h); }
        } else {
            if (g == 0) { j.kind = J_FWD; j.epi = X_B1; j.src = halo + 3 * N; j.slot = sB1(h); j.row = h; }
            else if (g == 2) { j.kind = J_FWD; j.epi = X_B3; j.src = halo + 4 * N; j.slot = sB3(h); j.row = h; }
        }
        return j;
    }
    const int r = (ri - 3) % 5;
    const int p = p0 + (ri - 3) / 5;
    if (p >= p1) return j;
    j.row = p;
    switch (r) {
    case 0:
        j.kind = J_FWD; j.epi = X_STORE;
        if (g == 0) { j.src = (p + 1 < p1) ? a.E[0] + (size_t)(p + 1) * N : halo + 5 * N; j.slot = sE1(p + 1); }
        else if (g == 1) { j.src = (p + 1 < p1) ? a.E[2] + (size_t)(p + 1) * N : halo + 6 * N; j.slot = sE3(p + 1); }
        else { j.src = a.E[1] + (size_t)p * N; j.slot = sE2; }
        break;
    case 1:
        j.kind = J_FWD;
        if (g == 0) { j.epi = X_B1; j.src = a.B[0] + (size_t)p * N; j.slot = sB1(p); }
        else if (g == 1) { j.epi = X_B2; j.src = a.B[1] + (size_t)p * N; j.slot = sB2; }
        else { j.epi = X_B3; j.src = a.B[2] + (size_t)p * N; j.slot = sB3(p); }
        break;
    case 2:
        j.kind = J_FWD;
        if (g == 0) { j.epi = X_J1; j.src = a.J[0] + (size_t)p * N; j.slot = sE1(p); }
        else if (g == 1) { j.epi = X_J2; j.src = a.J[1] + (size_t)p * N; j.slot = sE2; }
        else { j.epi = X_J3; j.src = a.J[2] + (size_t)p * N; j.slot = sE3(p); }
        break;
    case 3:
        j.kind = J_INV;
        if (g == 0) { j.slot = sE1(p); j.dst = a.E[0] + (size_t)p * N; }
        else if (g == 1) { j.slot = sE2; j.dst = a.E[1] + (size_t)p * N; }
        else { j.slot = sE3(p); j.dst = a.E[2] + (size_t)p * N; }
        break;
    default:
        j.kind = J_INV;
        if (g == 0) { j.slot = sB1(p); j.dst = a.B[0] + (size_t)p * N; }
        else if (g == 1) { j.slot = sB2; j.dst = a.B[1] + (size_t)p * N; }
        else { j.slot = sB3(p); j.dst = a.B[2] + (size_t)p * N; }
        break;
    }
    return j;
}

// source row of the idx-th forward transform of group g in a work item
// (prologue: P1 all groups, P2 groups 0 and 1, P3 groups 0 and 2; then R1, R2, R3 per row).
// Halo-buffer mode: rows outside the strip come from the buffer filled by k_halo.
// Flag mode: the row before the strip is read from the fields directly, and the
// row after it (E1, E3 only) from the copy published by the next strip.
__device__ __forceinline__ const float* fwd_src(const FusedInst& a, int N, int strip, int p0, int p1, int g, int idx,
                                                bool fm, int next) {
    const float* halo = a.halo + (size_t)strip * 7 * N;
    const int npro = (g == 0) ? 3 : 2;
    if (idx < npro) {
        if (fm) {
            const int h = (p0 - 1 + a.n2) % a.n2;
            if (idx == 0) return g == 0 ? a.E[0] + (size_t)p0 * N : g == 1 ? a.E[2] + (size_t)p0 * N : a.E[1] + (size_t)h * N;
            if (idx == 1) return g == 0 ? a.E[0] + (size_t)h * N : g == 1 ? a.E[2] + (size_t)h * N : a.B[2] + (size_t)h * N;
            return a.B[0] + (size_t)h * N;                                  // g == 0, P3
        }
        if (idx == 0) return g == 0 ? a.E[0] + (size_t)p0 * N : g == 1 ? a.E[2] + (size_t)p0 * N : halo + 1 * N;
        if (idx == 1) return g == 0 ? halo + 0 * N : g == 1 ? halo + 2 * N : halo + 4 * N;
        return halo + 3 * N;                                                // g == 0, P3
    }
    const int q = idx - npro;
    const int p = p0 + q / 3, r = q % 3;
    if (p >= p1) return nullptr;
    if (r == 0) {
        if (g == 2) return a.E[1] + (size_t)p * N;
        const int c = g == 0 ? 0 : 2;
        if (p + 1 < p1) return a.E[c] + (size_t)(p + 1) * N;
        if (fm) return a.halo + (size_t)next * 7 * N + (g == 0 ? 0 : 1) * N;
        return halo + (g == 0 ? 5 : 6) * N;
    }
    if (r == 1) return a.B[g] + (size_t)p * N;
    return a.J[g] + (size_t)p * N;
}


}  // namespace hyb
