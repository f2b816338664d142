// q3d_body.cuh -- device parts of the quasi-3D step shared by its kernels (quasi3d.cu) and the
// single-launch batched step (batch_step.cu): the per-mode tables, the 2048-point z transform of
// a row (next row in registers, or staged by bulk copy inside the single launch), and the
// leapfrog, per (axial mode, radial row) or per column of radial rows.
#pragma once
#include <math.h>

#include "hyb_internal.cuh"
#include "packed_dev.cuh"
#include "tm_dev.cuh"

namespace hyb {

template <typename T>
struct QTab {
    cplx<T> sp;   // sigma+ = i k e^{+i k dz/2}
    cplx<T> sm;   // sigma- = i k e^{-i k dz/2}
    T cjz;        // ampere dt F corr
    T cj;         // ampere dt F
};

// the arrays of up to kQModes modes advanced by one launch (modes of equal nz = 2048, nr, dr):
// mode q's field f at p[9 q + f], its spectra at spec[q]
constexpr int kQModes = 8;
struct QMulti { void* p[kQModes * 9]; float2* spec[kQModes]; int nm; };

constexpr int kQThreads = 256;

// ---------------------------------------------------------------- nz = 2048, FP32: register-resident rows
// X[k] = sum_j x[j] W^{jk}, W = exp(-2 pi i / 2048), factored 8 x 8 x 8 x 4 with k = k1 + 8 k2 + 64 k3 + 512 k4:
//   S1  thread t:            DFT8 over n of x[t + 256 n] -> k1, times W_2048^{t k1}      -> A(k1, t)
//   S2  (t0, k1) = (t & 31, t >> 5):  DFT8 over t1 of A(k1, t0 + 32 t1) -> k2, times W_256^{t0 k2}
//   S3  (u0, k1, k2) = (t & 3, (t >> 2) & 7, t >> 5):  DFT8 over u1 of A'(k1, k2, u0 + 4 u1) -> k3,
//       times W_32^{u0 k3}
//   S4  the 512 (k1, k2, k3) in two halves:  DFT4 over u0 -> k4, written to X[k1 + 8 k2 + 64 k3 + 512 k4]
// Exchange layouts (float2 units): A(k1, t) at 256 k1 + t; A'(k1, k2, t0) at 260 k1 + 32 k2 + t0;
// A''(k1, k2, k3, u0) at 516 u0 + 64 k3 + k1 + 8 k2 (in the A buffer).  With 8-byte accesses a half-warp
// of every exchange reaches 16 different bank pairs; global loads and stores are row-contiguous per warp.
// The inverse uses the conjugate twiddles and scales by 1/2048.  One row per 256-thread block
// iteration; persistent, the next row's points on their way (registers, or a bulk copy) while the
// current one is transformed.
constexpr int kQ2k = 2048;
constexpr int kQ2kA = 2064, kQ2kB = 2080;
constexpr int kQ2kTw = 7 * 256 + 7 * 32 + 7 * 4;     // stage twiddles, in the order the threads read them

template <bool INV>
__device__ __forceinline__ float2 q2k_tw(float2 a, float2 w) {
    return INV ? make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y))
               : make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// inside the single-launch batched step: a part's staging row (kQ2k float2 of shared memory) that
// the bulk-copy engine fills with the next row, the mbarrier (count 1, phase 0 at the start) it
// completes, and where a wait that gives up reports (bounded waits, as in the 2D kernels)
struct QStage { float2* stg; uint32_t bar; int* err; volatile int* abort; };

// One 256-thread block transforming rows vb, vb + vg, ... of io (thread t, exchange buffers bufA
// of kQ2kA and bufB of kQ2kB float2).  Standalone (MEGA = false) the block is a CTA and holds the
// next row in registers while it transforms the current one; inside the single-launch batched step
// it is one of the three 256-thread parts of a CTA (80 registers a thread), synchronised by named
// barrier bar_id, and the next row arrives by bulk copy into the staging row of qs.
template <bool INV, bool MEGA>
__device__ __forceinline__ void cfft2048_body(const QMulti& io, int nr, int nf, const float2* __restrict__ tw,
                                              int64_t vb, int64_t vg, int t, float2* bufA, float2* bufB, int bar_id,
                                              const QStage& qs = QStage{}) {
    auto bsync = [&]() {
        if constexpr (MEGA) asm volatile("bar.sync %0, 256;" :: "r"(bar_id) : "memory");
        else __syncthreads();
    };
    const int64_t per = (int64_t)nr * nf, total = per * io.nm;
    // stage twiddles: held in registers by a whole CTA of 256 threads; inside the single launch (80
    // registers a thread) read from the table when used, which the caller has put in shared memory
    float2 w1[8], w2[8], w3[8], nx[8];
    if constexpr (!MEGA) {
#pragma unroll
        for (int k = 1; k < 8; k++) {
            w1[k] = tw[(k - 1) * 256 + t];
            w2[k] = tw[1792 + (k - 1) * 32 + (t & 31)];
            w3[k] = tw[2016 + (k - 1) * 4 + (t & 3)];
        }
    }
    auto twid = [&](int s, int k) -> float2 {
        if constexpr (MEGA) {
            return s == 1 ? tw[(k - 1) * 256 + t] : s == 2 ? tw[1792 + (k - 1) * 32 + (t & 31)] : tw[2016 + (k - 1) * 4 + (t & 3)];
        } else {
            return s == 1 ? w1[k] : s == 2 ? w2[k] : w3[k];
        }
    };
    // row j of the launch: mode q, field f, radial row r; its spectrum row is jj of mode q
    auto src_of = [&](int64_t j) -> const float2* {
        const int q = (int)(j / per);
        const int64_t jj = j - q * per;
        const int f = (int)(jj / nr);
        const int64_t r = jj - (int64_t)f * nr;
        return INV ? io.spec[q] + jj * kQ2k : reinterpret_cast<const float2*>(io.p[9 * q + f]) + r * kQ2k;
    };
    auto fetch = [&](int64_t j) {
        const float2* x = src_of(j);
#pragma unroll
        for (int n = 0; n < 8; n++) nx[n] = __ldcs(x + t + 256 * n);
    };
    // MEGA: the bulk copy of row jn into the staging row (thread 0, after the part's reads of it)
    uint32_t ph = 0;
    bool pending = false;
    auto stage = [&](int64_t jn) {
        if (t == 0) {
            fence_proxy_async_smem();
            mbar_expect_tx(qs.bar, kQ2k * 8);
            bulk_load(smem_addr(qs.stg), src_of(jn), kQ2k * 8, qs.bar);
        }
        pending = true;
    };
    int64_t j = vb;
    if (j < total) {
        if constexpr (MEGA) stage(j);
        else fetch(j);
    }
    for (; j < total; j += vg) {
        float2 v[8];
        if constexpr (MEGA) {
            mbar_wait(qs.bar, ph, qs.err, qs.abort);
            ph ^= 1;
            pending = false;
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = qs.stg[t + 256 * n];
        } else {
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = nx[n];
            if (j + vg < total) fetch(j + vg);
        }
        // S1
        dft8x<INV>(v);
#pragma unroll
        for (int k = 1; k < 8; k++) v[k] = q2k_tw<INV>(v[k], twid(1, k));
        bsync();                 // the previous row's S4 has read the A buffer (MEGA: all have read the staging row)
        if constexpr (MEGA) {
            if (j + vg < total) stage(j + vg);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) bufA[256 * k + t] = v[k];
        bsync();
        // S2
        {
            const int t0 = t & 31, k1 = t >> 5;
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = bufA[256 * k1 + t0 + 32 * n];
            dft8x<INV>(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = q2k_tw<INV>(v[k], twid(2, k));
#pragma unroll
            for (int k = 0; k < 8; k++) bufB[260 * k1 + 32 * k + t0] = v[k];
        }
        bsync();
        // S3
        {
            const int u0 = t & 3, k1 = (t >> 2) & 7, k2 = t >> 5;
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = bufB[260 * k1 + 32 * k2 + u0 + 4 * n];
            dft8x<INV>(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = q2k_tw<INV>(v[k], twid(3, k));
#pragma unroll
            for (int k = 0; k < 8; k++) bufA[516 * u0 + 64 * k + k1 + 8 * k2] = v[k];
        }
        bsync();
        // S4
        float2* X;
        {
            const int q = (int)(j / per);
            const int64_t jj = j - q * per;
            const int f = (int)(jj / nr);
            const int64_t r = jj - (int64_t)f * nr;
            X = INV ? reinterpret_cast<float2*>(io.p[9 * q + f]) + r * kQ2k : io.spec[q] + jj * kQ2k;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int it = t + 256 * h;      // k1 + 8 k2 + 64 k3
            float2 a0 = bufA[it], a1 = bufA[516 + it], a2 = bufA[1032 + it], a3 = bufA[1548 + it];
            dft4x<INV>(a0, a1, a2, a3);
            if (INV) {
                const float s = 1.0f / (float)kQ2k;
                a0 = vmul(a0, make_float2(s, s)); a1 = vmul(a1, make_float2(s, s));
                a2 = vmul(a2, make_float2(s, s)); a3 = vmul(a3, make_float2(s, s));
            }
            __stcs(X + it, a0);
            __stcs(X + it + 512, a1);
            __stcs(X + it + 1024, a2);
            __stcs(X + it + 1536, a3);
        }
    }
    // a bulk copy still in flight (only after a wait that gave up) lands before the part moves on
    if constexpr (MEGA) {
        if (pending && t == 0) mbar_drain(qs.bar, ph);
    }
}

template <typename T>
struct QB { cplx<T> z, r, p; };

// complex arithmetic of the leapfrog with every operation rounded on its own (never contracted into
// an FMA), so that the one-point and the column forms, inlined into different kernels, give the
// same bits
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
template <typename C> __device__ __forceinline__ C qadd(C a, C b) { return mkc<C>(rn_add(a.x, b.x), rn_add(a.y, b.y)); }
template <typename C> __device__ __forceinline__ C qsub(C a, C b) { return mkc<C>(rn_sub(a.x, b.x), rn_sub(a.y, b.y)); }
template <typename C> __device__ __forceinline__ C qmul(C a, C b) {
    return mkc<C>(rn_sub(rn_mul(a.x, b.x), rn_mul(a.y, b.y)), rn_add(rn_mul(a.x, b.y), rn_mul(a.y, b.x)));
}
template <typename C> __device__ __forceinline__ C qscale(C a, decltype(C::x) s) { return mkc<C>(rn_mul(a.x, s), rn_mul(a.y, s)); }
// i m / r times a
template <typename C> __device__ __forceinline__ C qimr(C a, decltype(C::x) m_over_r) {
    return mkc<C>(rn_mul(-m_over_r, a.y), rn_mul(m_over_r, a.x));
}

// Faraday for axial mode k at radial row j: B^{n+1/2} from B^{n-1/2} at j and E^n at rows j and j+1
// (tangential E vanishes on the conducting wall r = nr dr, so E at row nr is 0; on the axis B_r
// follows the m rules, for m = 1 with E_z at row 1, which is row j + 1 there)
template <typename T>
__device__ __forceinline__ QB<T> qfaraday(cplx<T> ez, cplx<T> er, cplx<T> ep, cplx<T> ezu, cplx<T> epu, cplx<T> bz,
                                          cplx<T> br, cplx<T> bp, int j, cplx<T> sp, T dt, T dr, int m) {
    using C = cplx<T>;
    const T ri = (T)j * dr, rh = ((T)j + (T)0.5) * dr, rup = (T)(j + 1) * dr;
    const T mT = (T)m;
    C cr;
    if (j > 0) cr = qsub(qimr(ez, mT / ri), qmul(sp, ep));
    else if (m == 1) cr = qsub(qimr(ezu, mT / dr), qmul(sp, ep));
    else cr = mkc<C>((T)0, (T)0);
    const C cp = qsub(qmul(sp, er), qscale(qsub(ezu, ez), (T)1 / dr));
    const C cz = qsub(qscale(qsub(qscale(epu, rup), qscale(ep, ri)), (T)1 / (rh * dr)), qimr(er, mT / rh));
    QB<T> b;
    b.z = qsub(bz, qscale(cz, dt));
    b.r = (j == 0 && m != 1) ? mkc<C>((T)0, (T)0) : qsub(br, qscale(cr, dt));
    b.p = qsub(bp, qscale(cp, dt));
    return b;
}

// the same with E and B read from the spectra [E, B, J] (field stride fs)
template <typename T>
__device__ __forceinline__ QB<T> qfaraday_at(const cplx<T>* __restrict__ spec, int64_t fs, int nz, int nr, int j, int k,
                                             cplx<T> sp, T dt, T dr, int m) {
    using C = cplx<T>;
    const C* Ez = spec; const C* Er = spec + fs; const C* Ep = spec + 2 * fs;
    const C* Bz = spec + 3 * fs; const C* Br = spec + 4 * fs; const C* Bp = spec + 5 * fs;
    const int64_t i = (int64_t)j * nz + k, iu = i + nz;
    const C ezu = (j + 1 < nr) ? Ez[iu] : mkc<C>((T)0, (T)0);
    const C epu = (j + 1 < nr) ? Ep[iu] : mkc<C>((T)0, (T)0);
    return qfaraday<T>(Ez[i], Er[i], Ep[i], ezu, epu, Bz[i], Br[i], Bp[i], j, sp, dt, dr, m);
}

// Ampere at row j from B^{n+1/2} at rows j (b) and j-1 (bd, unused at j = 0), E^n and j at row j:
// E^{n+1} (z, r, phi); on the axis E_z only for m = 0, E_phi only for m = 1
template <typename T>
__device__ __forceinline__ QB<T> qampere(const QB<T>& b, const QB<T>& bd, cplx<T> ez, cplx<T> er, cplx<T> ep, cplx<T> jz,
                                         cplx<T> jr, cplx<T> jp, const QTab<T>& q, int j, T dt, T dr, int m) {
    using C = cplx<T>;
    const T ri = (T)j * dr, rh = ((T)j + (T)0.5) * dr, rd = ((T)j - (T)0.5) * dr;
    const T mT = (T)m;
    const C cr = qsub(qimr(b.z, mT / rh), qmul(q.sm, b.p));
    C cp, cz;
    if (j > 0) {
        cp = qsub(qmul(q.sm, b.r), qscale(qsub(b.z, bd.z), (T)1 / dr));
        cz = qsub(qscale(qsub(qscale(b.p, rh), qscale(bd.p, rd)), (T)1 / (ri * dr)), qimr(b.r, mT / ri));
    } else {
        cp = (m == 1) ? qsub(qmul(q.sm, b.r), qscale(b.z, (T)2 / dr)) : mkc<C>((T)0, (T)0);
        cz = (m == 0) ? qscale(b.p, (T)4 / dr) : mkc<C>((T)0, (T)0);
    }
    QB<T> e;
    e.r = qsub(qadd(er, qscale(cr, dt)), qscale(jr, q.cj));
    e.p = qsub(qadd(ep, qscale(cp, dt)), qscale(jp, q.cj));
    e.z = qsub(qadd(ez, qscale(cz, dt)), qscale(jz, q.cjz));
    if (j == 0 && m != 0) e.z = mkc<C>((T)0, (T)0);
    if (j == 0 && m != 1) e.p = mkc<C>((T)0, (T)0);
    return e;
}

// one leapfrog step per (axial mode k, radial row j) on the spectra [E, B, J] (slots 0..8): Faraday at
// rows j and j-1 (the latter recomputed, so no launch boundary is needed between the halves), then
// Ampere at row j.  E^{n+1} goes to the J slots 6..8 (J at row j is read by this thread only) and
// B^{n+1/2} to slots 9..11; slots 0..5 are only read, so neighbouring threads see the old values.
template <typename T>
struct QLeap { cplx<T>* spec[kQModes]; const QTab<T>* tab[kQModes]; T dt[kQModes]; int m[kQModes]; };

// axial mode k of radial row j of mode qm
template <typename T>
__device__ __forceinline__ void qleap_body(const QLeap<T>& ql, int nz, int nr, T dr, int k, int j, int qm) {
    using C = cplx<T>;
    cplx<T>* __restrict__ spec = ql.spec[qm];
    const QTab<T>* __restrict__ tab = ql.tab[qm];
    const T dt = ql.dt[qm];
    const int m = ql.m[qm];
    if (k >= nz) return;
    const int64_t fs = (int64_t)nr * nz, i = (int64_t)j * nz + k;
    const C* Ez = spec; const C* Er = spec + fs; const C* Ep = spec + 2 * fs;
    C* Jz = spec + 6 * fs; C* Jr = spec + 7 * fs; C* Jp = spec + 8 * fs;
    C* Bn = spec + 9 * fs;
    const QTab<T> q = tab[k];
    const QB<T> b = qfaraday_at<T>(spec, fs, nz, nr, j, k, q.sp, dt, dr, m);
    QB<T> bd = b;
    if (j > 0) bd = qfaraday_at<T>(spec, fs, nz, nr, j - 1, k, q.sp, dt, dr, m);
    const QB<T> e = qampere<T>(b, bd, Ez[i], Er[i], Ep[i], Jz[i], Jr[i], Jp[i], q, j, dt, dr, m);
    Jz[i] = e.z;
    Jr[i] = e.r;
    Jp[i] = e.p;
    Bn[i] = b.z;
    Bn[fs + i] = b.r;
    Bn[2 * fs + i] = b.p;
}

// The same for rows j0 .. j1 - 1 of the 256 axial modes kb * 256 .. + 255 of mode qm, one per thread
// t of a 256-thread part of a CTA (80 registers a thread, inside the single-launch batched step),
// sweeping up the radius.  E at row j and B^{n+1/2} at row j - 1 are carried in registers from row
// to row; E at row j + 1 and B, j at row j arrive by bulk copy (nine 2 KB row segments, one stage)
// into one of two stage buffers of st (2 x 9 x 256 complex, shared memory) two rows ahead, so that
// every value is read once and the loads in flight do not take registers.  bar0, bar1: the two
// stages' mbarriers (count 1); bit b of phases: the parity buffer b waits for next, bit 2 + b: buffer
// b has been used; bar_id: the part's named barrier.
template <typename T>
__device__ __forceinline__ void qleap_column(const QLeap<T>& ql, int nz, int nr, T dr, int kb, int qm, int j0, int j1,
                                             int t, cplx<T>* st, uint32_t bar0, uint32_t bar1, uint32_t& phases,
                                             int bar_id, int* err, volatile int* abort) {
    using C = cplx<T>;
    cplx<T>* __restrict__ spec = ql.spec[qm];
    const T dt = ql.dt[qm];
    const int m = ql.m[qm];
    const int64_t fs = (int64_t)nr * nz;
    const int k = kb * 256 + t;
    C* Jz = spec + 6 * fs; C* Jr = spec + 7 * fs; C* Jp = spec + 8 * fs;
    C* Bn = spec + 9 * fs;
    const C zero = mkc<C>((T)0, (T)0);
    const QTab<T> q = ql.tab[qm][k];
    constexpr uint32_t SEG = 256 * sizeof(C);
    // stage of row r into buffer b: E (slots 0..2) at row r + 1 (none past the wall), B (3..5) and j
    // (6..8) at row r
    auto stage = [&](int r, int b) {
        if (t == 0) {
            fence_proxy_async_smem();
            const bool e_up = r + 1 < nr;
            const uint32_t bar = b ? bar1 : bar0;
            mbar_expect_tx(bar, (e_up ? 9u : 6u) * SEG);
            C* dst = st + b * 9 * 256;
            for (int f = 0; f < 9; f++) {
                if (f < 3 && !e_up) continue;
                const int row = f < 3 ? r + 1 : r;
                bulk_load(smem_addr(dst + f * 256), spec + f * fs + (int64_t)row * nz + kb * 256, SEG, bar);
            }
        }
        phases |= 4u << b;
    };
    // E at row j0 and B^{n+1/2} at row j0 - 1 from memory
    int64_t i = (int64_t)j0 * nz + k;
    C ez = spec[i], er = spec[fs + i], ep = spec[2 * fs + i];
    QB<T> bd = {zero, zero, zero};
    if (j0 > 0) {
        const int64_t id = i - nz;
        bd = qfaraday<T>(spec[id], spec[fs + id], spec[2 * fs + id], ez, ep, spec[3 * fs + id], spec[4 * fs + id],
                         spec[5 * fs + id], j0 - 1, q.sp, dt, dr, m);
    }
    stage(j0, 0);
    if (j0 + 1 < j1) stage(j0 + 1, 1);
    for (int j = j0; j < j1; j++) {
        const int b = (j - j0) & 1;
        mbar_wait(b ? bar1 : bar0, (phases >> b) & 1u, err, abort);
        phases ^= 1u << b;
        const C* sb = st + b * 9 * 256 + t;
        const bool e_up = j + 1 < nr;
        const C ezu = e_up ? sb[0] : zero, eru = e_up ? sb[256] : zero, epu = e_up ? sb[512] : zero;
        const C bz = sb[768], br = sb[1024], bp = sb[1280], jz = sb[1536], jr = sb[1792], jp = sb[2048];
        asm volatile("bar.sync %0, 256;" :: "r"(bar_id) : "memory");      // the part has read the buffer
        if (j + 2 < j1) stage(j + 2, b);
        const QB<T> bn = qfaraday<T>(ez, er, ep, ezu, epu, bz, br, bp, j, q.sp, dt, dr, m);
        const QB<T> e = qampere<T>(bn, bd, ez, er, ep, jz, jr, jp, q, j, dt, dr, m);
        Jz[i] = e.z;
        Jr[i] = e.r;
        Jp[i] = e.p;
        Bn[i] = bn.z;
        Bn[fs + i] = bn.r;
        Bn[2 * fs + i] = bn.p;
        bd = bn;
        ez = ezu; er = eru; ep = epu;
        i += nz;
    }
}

// everything the three quasi-3D stages of up to kQModes FP32 modes with nz = 2048 need
struct Q3Args {
    QMulti fin, fout;          // forward: the nine arrays of each mode; inverse: its six advanced spectra
    QLeap<float> ql;
    const float2* tw2k;
    int nr, nm;
    float dr;
};
hyb_status quasi3d_step_args(hyb_grid* const* gs, int n, Q3Args* out);

}  // namespace hyb
