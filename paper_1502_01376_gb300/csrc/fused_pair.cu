// fused_pair.cu -- single-pass FP32 hybrid advance for n1 = 4096 with the
// fields transformed in pairs (one strip of x2 rows per CTA, all CTAs
// co-resident, halo rows exchanged in the kernel through flags).
//
// Arithmetic (Eqs. hybrid2db1-hybrid2de3 with Eq. currentcorrection and the
// Sec. 4 filter folded into the current coefficients cj1, cj):
//   k1 space, per mode:  B2' = B2 + S E3                    S = c dt sigma+
//                        B3' = B3 + a2 (E1(p+1) - E1(p)) - S E2
//                        E1' = E1 + a2 (B3'(p) - B3'(p-1)) - cj1 j1
//                        E2' = E2 + conj(S) B3' - cj j2
//                        E3' = E3 - conj(S) B2' - cj j3      (all rows' sums, a2 = c dt / dx2)
//   real space:          B1' = B1 - a2 (E3(p+1) - E3(p))
//                        E3  <- E3' - a2 (B1'(p) - B1'(p-1))
// B1 carries no x1 derivative and E3's x2 difference of B1 is linear, so both
// are applied in real space (the same result up to rounding): a row needs 8
// forward and 5 inverse transforms instead of 9 and 6.
//
// Two real rows f0, f1 are transformed together as the complex row
// z = f0 + i f1 (4096 points), z -> Z by three radix-16 stages
//   S1  thread s = n1 + 16 n2 holds z[s + 256 n3]; 16-point DFT over n3 -> k1;
//       twiddle W_4096^(s k1)
//   S2  thread (n1, k1): 16-point DFT over n2 -> k2; twiddle W_256^(n1 k2)
//   S3  thread of column c = k1 + 16 k2: 16-point DFT over n1 -> Z[c + 256 k3]
// and separated, F0[k] = (Z[k] + conj Z[N-k]) / 2, F1[k] = (Z[k] - conj Z[N-k]) / 2i.
// Columns c and 256 - c sit in the two lanes of a lane pair, which swap the
// upper half of their outputs (shuffle) so that each thread ends up owning
// the modes k = c + 256 q, q = 0..7, of both fields (column 0 also owns the
// Nyquist mode, packed with mode 0 as both are real).  k1-space values are
// kept doubled (2F); the inverse scales by 1/(2 N).
//
// A CTA has two groups of 256 threads.  A strip's work is a list of jobs,
// each a pair of transforms (or an epilogue alone), split between the groups
// by a list schedule the host computes from the jobs' dependencies and costs;
// a group runs its list in order and, before a job that reads what the other
// group writes, waits for that job's done flag in shared memory:
//   P1  F(E1(p0), E1(p0-1))            P2  F(E2(p0-1), B3(p0-1))
//   P3  B3'(p0-1) from P1, P2; B1'(p0-1)            (the strip's prologue)
//   A   F(E2, E3)(p)          -> slot EA(p)
//   B   F(E1(p+1), j1(p))     -> slot EB(p)
//   C   F(B2, B3)(p) + B2', B3'               -> slot BC(p)
//   D   F(j2, j3)(p) + E2', E3' -> EA(p); E1'(p) -> EB(p) in place of j1
//   E   inverse EA(p) -> E2, E3 (minus the B1' difference)
//   F   inverse BC(p) -> B2, B3
//   G   inverse EB(p) -> E1 (its second row); B1'(p) in real space
// The k1-space slots live in tensor memory: thread s of either group owns the
// same modes and keeps them in TMEM lane s mod 128, so a job's epilogue reads
// any other job's slots lane-locally.  Input rows of forward jobs arrive by
// bulk copy (cp.async.bulk) into the group's staging buffer, one forward job
// ahead.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "fused_api.cuh"
#include "fused_dev.cuh"
#include "packed_dev.cuh"
#include "tm_dev.cuh"

namespace hyb {

namespace pq {
constexpr int N = 4096;
constexpr int T = 256;                         // threads per group
constexpr int G = 2;                           // groups
constexpr int NT = G * T;
constexpr int OFF_STAGE = 0;                   // [G][2][N] float
constexpr int XS = 4368;                                // exchange buffer (float2), padded rows of 17
constexpr int OFF_X = OFF_STAGE + G * 2 * N * 4;        // [G][2][XS] float2: X1, X2
constexpr int OFF_B1 = OFF_X + G * 2 * XS * 8;          // [N] float: B1' of the last row updated
constexpr int OFF_TW2 = OFF_B1 + N * 4;                 // [16][16] float2: W_256^(n1 k2)
constexpr int OFF_SYMN = OFF_TW2 + 16 * 16 * 8;         // float4: Nyquist {S, -, cj1, cj}
constexpr int OFF_BAR = OFF_SYMN + 16;                  // [G] mbarrier
constexpr int OFF_MISC = OFF_BAR + G * 8;               // TMEM base, abort flag
constexpr int MAXR = 64;                                // schedule rounds
constexpr int OFF_DONE = OFF_MISC + 16;                 // [G][MAXR] int: job of (group, round) done
constexpr int SMEM = OFF_DONE + G * MAXR * 4;
constexpr uint32_t TMEM_COLS = 512;
constexpr int COL_SYM = 384;                   // per thread 32 words: {Sx, Sy, cj1, cj} of 8 modes
constexpr int COL_TW = 448;                    // per thread 30 words: W_4096^(s k), k = 1..15
constexpr float INV2N = 1.0f / 8192.0f;
}  // namespace pq

// job kinds and round flags of the schedule
enum : int { PJ_IDLE = 0, PJ_A, PJ_B, PJ_C, PJ_D, PJ_E, PJ_F, PJ_G, PJ_P1, PJ_P2, PJ_P3 };
enum : int { PF_WAIT_PUB = 1, PF_WAIT_READ = 2, PF_SET_PUB = 4, PF_SET_READ = 8 };
// one entry of a group's job list: kind, strip-relative row, flags, synchronisation (bit 0:
// wait for dependencies or a flag first; bit 1: a group barrier and the done flag afterwards),
// and the positions in the other group's list of the jobs it waits for (bit q: position q)
enum : int { PS_START = 1, PS_END = 2 };
struct PJob { int8_t job; int8_t row; uint8_t flags; uint8_t sync; int pad; unsigned long long dep; };

struct PairArgs {
    FusedInst a;
    const int4* items;            // {0, strip, p0, p1} per CTA
    const PJob* sched[2];         // job lists [G][nrounds] for strip heights hs[0], hs[1]
    int nrounds[2];
    int hs[2];
    const float2* tw;             // W_4096^j, j < 4096
    float* scratch;               // [strips][2][N]: a2 (B1'(p) - B1'(p-1)) by row parity
    int* flags;                   // [2 strips]: published, read
    int epoch;
    int n_strips;
    int* err;
};

// ------------------------------------------------------------------ 16-point DFTs on (re, im) pairs
// radix 4 x 4: n = 4 a + b, k = k1 + 4 k2; DFT4 over a, twiddle W16^(b k1), DFT4 over b
template <bool INV>
__device__ __forceinline__ float2 w16mul(float2 v, int e) {
    // v W16^e (conjugate root for INV), e known after unrolling
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
    const int j = e & 15;
    float c, s;          // W16^j = c - i s (forward)
    switch (j) {
    case 0: return v;
    case 1: c = c1; s = s1; break;
    case 2: c = h; s = h; break;
    case 3: c = s1; s = c1; break;
    case 4: return INV ? f2(-v.y, v.x) : f2(v.y, -v.x);
    case 6: c = -h; s = h; break;
    case 9: c = -c1; s = -s1; break;
    default: c = 1.f; s = 0.f; break;
    }
    if (INV) s = -s;
    // (v.x + i v.y)(c - i s) = (v.x c + v.y s) + i (v.y c - v.x s)
    return f2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
}

template <bool INV>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
    float2 y[4][4];
#pragma unroll
    for (int b = 0; b < 4; b++) {
        y[b][0] = x[b]; y[b][1] = x[4 + b]; y[b][2] = x[8 + b]; y[b][3] = x[12 + b];
        dft4x<INV>(y[b][0], y[b][1], y[b][2], y[b][3]);
    }
#pragma unroll
    for (int b = 1; b < 4; b++)
#pragma unroll
        for (int k1 = 1; k1 < 4; k1++) y[b][k1] = w16mul<INV>(y[b][k1], b * k1);
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
        float2 p = y[0][k1], q = y[1][k1], r = y[2][k1], t = y[3][k1];
        dft4x<INV>(p, q, r, t);
        x[k1] = p; x[k1 + 4] = q; x[k1 + 8] = r; x[k1 + 12] = t;
    }
}

// ------------------------------------------------------------------ index maps
// exchange 1 (S1 -> S2): element (n1, k1, n2) at 273 n1 + 17 k1 + n2; exchange 2 (S2 -> S3):
// element (column c, n1) at 17 P(c) + n1, P(c) = c below 128 and 128 + ((264 - c) mod 128) above,
// so that the columns c and 256 - c of a lane pair fall in different bank pairs.  Both sides of
// both exchanges address affinely in their loop index (immediate offsets), and the 16 lanes of a
// half warp (128 bytes of 8-byte elements) always hit 16 different bank pairs.
__device__ __forceinline__ int x1pos(int n1, int k1, int n2) { return 273 * n1 + 17 * k1 + n2; }
__device__ __forceinline__ int pcol(int c) { return c < 128 ? c : 128 + ((264 - c) & 127); }
__device__ __forceinline__ int x2pos(int c, int n1) { return 17 * pcol(c) + n1; }
// S3 column of group thread s: lanes 2i, 2i + 1 of warp w hold columns j, 256 - j (j = 16 w + i),
// except lanes 0, 1 of warp 0, which hold the self-paired columns 0 and 128
__device__ __forceinline__ int col_of(int s) {
    const int w = s >> 5, l = s & 31, i = l >> 1, b = l & 1;
    if (w == 0 && i == 0) return b ? 128 : 0;
    const int j = 16 * w + i;
    return b ? 256 - j : j;
}

// TMEM address of this thread's words: lane s mod 128 (the warp's lane quarter), column base
__device__ __forceinline__ uint32_t tm_thread(uint32_t tbase, int s) {
    return tbase + ((uint32_t)(s & 127) << 16) + (uint32_t)((s >> 7) * 32);
}

// ------------------------------------------------------------------ the kernel
__global__ void __launch_bounds__(pq::NT, 1) k_fused_pair(PairArgs P) {
    using namespace pq;
    extern __shared__ __align__(128) unsigned char sm[];
    float* stage = reinterpret_cast<float*>(sm + OFF_STAGE);
    float2* xb = reinterpret_cast<float2*>(sm + OFF_X);
    float* b1s = reinterpret_cast<float*>(sm + OFF_B1);
    volatile int* done = reinterpret_cast<volatile int*>(sm + OFF_DONE);
    float2* tw2 = reinterpret_cast<float2*>(sm + OFF_TW2);
    float4* symN = reinterpret_cast<float4*>(sm + OFF_SYMN);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(sm + OFF_MISC);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + OFF_MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid / T, s = tid % T;
    const FusedInst& a = P.a;
    const int4 it = P.items[blockIdx.x];
    const int strip = it.y, p0 = it.z, p1 = it.w, H = p1 - p0;
    const int n2 = a.n2;
    const int next = (strip + 1) % P.n_strips;
    const int si = (H == P.hs[0]) ? 0 : 1;
    const PJob* sched = P.sched[si] + g * P.nrounds[si];     // this group's job list
    const int R = P.nrounds[si];
    const float a2 = a.a2;

    // ---- set-up: TMEM, barriers, tables
    if (warp == 0) {
        tm_alloc(smem_addr(s_taddr), TMEM_COLS);
        tm_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < G; k++) mbar_init(smem_addr(bars + k), 1);
        mbar_fence_init();
        *s_abort = 0;
        *symN = a.sym[2048];
    }
    for (int i = tid; i < G * MAXR; i += NT) done[i] = 0;
    for (int i = tid; i < 256; i += NT) {              // W_256^(n1 k2) = W_4096^(16 n1 k2)
        const int n1 = i & 15, k2 = i >> 4;
        tw2[k2 * 16 + n1] = P.tw[(16 * n1 * k2) & (N - 1)];
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = *s_taddr;
    const uint32_t tt = tm_thread(tbase, s);
    const int c = col_of(s);
    if (g == 0) {
        // per-thread twiddles W_4096^(s k), k = 1..15, and the symbols of this thread's modes
        float r[32];
#pragma unroll
        for (int k = 1; k < 16; k++) {
            const float2 w = P.tw[(s * k) & (N - 1)];
            r[2 * k - 2] = w.x;
            r[2 * k - 1] = w.y;
        }
        r[30] = 0.f;
        r[31] = 0.f;
        tm_st16_at<0>(tt + COL_TW, r);
        tm_st16_at<16>(tt + COL_TW + 16, r);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            float4 v = a.sym[c + 256 * q];
            if (c == 0 && q == 0) v = make_float4(0.f, 0.f, v.z, v.w);     // the packed DC / Nyquist mode
            r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
        }
        tm_st16_at<0>(tt + COL_SYM, r);
        tm_st16_at<16>(tt + COL_SYM + 16, r);
        tm_wait_st();
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();

    const uint32_t bar = smem_addr(bars + g);
    float* stg = stage + g * 2 * N;
    float2* X1 = xb + (g * 2 + 0) * XS;
    float2* X2 = xb + (g * 2 + 1) * XS;
    uint32_t nld = 0;                    // bulk loads of this group consumed (mbarrier phase)
    bool pending = false;                // a staged load issued and not yet consumed
    int staged_round = -1;               // round of the job whose rows are being staged
    const bool special = (s < 2);        // columns 0 and 128 (self-paired)

    auto rowp = [&](int rr) { return (p0 + rr + n2) % n2; };              // absolute row of strip-relative rr
    auto slot_col = [&](int kind, int rr) {                               // TMEM column of a pair slot
        const int par = (rr + 2) & 1;
        return (uint32_t)(64 * (2 * kind + par));                         // kind 0: EA, 1: EB, 2: BC
    };
    // source rows of a forward job (f0, f1)
    auto fwd_src = [&](int job, int rr, const float** f0, const float** f1) {
        const int p = rowp(rr);
        const float* halo_next = a.halo + (size_t)next * 7 * N;
        switch (job) {
        case PJ_A: *f0 = a.E[1] + (size_t)p * N; *f1 = a.E[2] + (size_t)p * N; break;
        case PJ_B: *f0 = (rr + 1 < H) ? a.E[0] + (size_t)rowp(rr + 1) * N : halo_next + 0 * N; *f1 = a.J[0] + (size_t)p * N; break;
        case PJ_C: *f0 = a.B[1] + (size_t)p * N; *f1 = a.B[2] + (size_t)p * N; break;
        case PJ_D: *f0 = a.J[1] + (size_t)p * N; *f1 = a.J[2] + (size_t)p * N; break;
        case PJ_P1: *f0 = a.E[0] + (size_t)rowp(0) * N; *f1 = a.E[0] + (size_t)rowp(-1) * N; break;
        default: *f0 = a.E[1] + (size_t)rowp(-1) * N; *f1 = a.B[2] + (size_t)rowp(-1) * N; break;   // P2
        }
    };
    auto is_fwd = [](int job) { return job == PJ_A || job == PJ_B || job == PJ_C || job == PJ_D || job == PJ_P1 || job == PJ_P2; };
    // the next forward job of this group after round r (its rows may be staged early unless it
    // reads a halo row another strip publishes: those are staged at the job's own start)
    auto next_fwd = [&](int r) {
        for (int q = r + 1; q < R; q++)
            if (is_fwd(sched[q].job)) return q;
        return -1;
    };
    // the last row's B job reads E1(p1) from the copy the next strip publishes: with plain loads
    // after the flag, not staged (only its j1 row is staged)
    auto direct0 = [&](int job, int rr) { return job == PJ_B && rr == H - 1; };
    auto issue_stage = [&](int q) {
        const int qj = sched[q].job, qr = sched[q].row;
        const float *f0, *f1;
        fwd_src(qj, qr, &f0, &f1);
        if (s == 0) {
            fence_proxy_async_smem();
            if (direct0(qj, qr)) {
                mbar_expect_tx(bar, 4 * N);
            } else {
                mbar_expect_tx(bar, 8 * N);
                bulk_load(smem_addr(stg), f0, 4 * N, bar);
            }
            bulk_load(smem_addr(stg + N), f1, 4 * N, bar);
        }
        pending = true;
        staged_round = q;
    };
    {
        const int q = next_fwd(-1);
        if (q >= 0) issue_stage(q);
    }

    auto gsync = [&]() { asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(T) : "memory"); };
    for (int r = 0; r < R; r++) {
        const PJob je = sched[r];
        const int job = je.job, rr = je.row, fl = je.flags, sy = je.sync;
        if (job == PJ_IDLE) continue;
        // wait for the other group's jobs this one reads from (bounded), and for the neighbour strip
        if (sy & PS_START) {
          if (s == 0) {
            unsigned long long m = je.dep;
            const long long t0 = clock64();
            while (m && !*s_abort) {
                const int q = __ffsll((long long)m) - 1;
                if (done[(1 - g) * MAXR + q]) { m &= m - 1; continue; }
                if (clock64() - t0 > kWaitCycles) { atomicOr(P.err, 2); *s_abort = 1; break; }
                __nanosleep(64);
            }
            __threadfence_block();
            if (fl & PF_WAIT_PUB) wait_flag(P.flags + 2 * next, P.epoch, P.err);
            if (fl & PF_WAIT_READ) wait_flag(P.flags + 2 * next + 1, P.epoch, P.err);
          }
          gsync();
          tm_fence_after();
        }
        if (is_fwd(job)) {
            if (staged_round != r) issue_stage(r);
            float b1v[16];
            if (job == PJ_A && s == 0)           // B1(p), which the next A job reads, into L2 now
                bulk_prefetch_l2(a.B[0] + (size_t)rowp(rr) * N, 4 * N);
            if (job == PJ_A && rr >= 1) {        // B1(p-1) + a2 E3(p-1), loaded while the rows land
                const float* b1 = a.B[0] + (size_t)rowp(rr - 1) * N;
                const float* e3 = a.E[2] + (size_t)rowp(rr - 1) * N;
#pragma unroll
                for (int n = 0; n < 16; n++) b1v[n] = fmaf(a2, e3[s + 256 * n], b1[s + 256 * n]);
            }
            mbar_wait(bar, nld & 1, P.err, s_abort);
            nld++;
            pending = false;
            // ---------------- S1: z[s + 256 n3], DFT16 over n3, twiddle W_4096^(s k1)
            float2 v[16];
            if (direct0(job, rr)) {
                const float* h = a.halo + (size_t)next * 7 * N;
#pragma unroll
                for (int n = 0; n < 16; n++) v[n] = f2(__ldcg(h + s + 256 * n), stg[N + s + 256 * n]);
            } else {
#pragma unroll
                for (int n = 0; n < 16; n++) v[n] = f2(stg[s + 256 * n], stg[N + s + 256 * n]);
            }
            if (job == PJ_P1) {                  // publish E1(p0) for the previous strip
                float* h = const_cast<float*>(a.halo) + (size_t)strip * 7 * N;
#pragma unroll
                for (int n = 0; n < 16; n++) h[s + 256 * n] = v[n].x;
                __threadfence();
            } else if (job == PJ_A) {
                if (rr == 0) {                   // publish E3(p0)
                    float* h = const_cast<float*>(a.halo) + ((size_t)strip * 7 + 1) * N;
#pragma unroll
                    for (int n = 0; n < 16; n++) h[s + 256 * n] = v[n].y;
                    __threadfence();
                } else {
                    // B1'(p-1) = B1(p-1) - a2 (E3(p) - E3(p-1)) in real space (E(p-1), which overwrites
                    // E3(p-1), waits for this job); out to B1, and a2 (B1'(p-1) - B1'(p-2)) to the
                    // scratch row of E(p-1)
                    float* dsc = P.scratch + ((size_t)strip * 2 + ((rr - 1) & 1)) * N;
                    float* b1o = a.B[0] + (size_t)rowp(rr - 1) * N;
#pragma unroll
                    for (int n = 0; n < 16; n++) {
                        const float b1n = b1v[n] - a2 * v[n].y;
                        __stcg(dsc + s + 256 * n, a2 * (b1n - b1s[s + 256 * n]));
                        b1s[s + 256 * n] = b1n;
                        stg_stream1(b1o + s + 256 * n, b1n);
                    }
                }
            }
            dft16<false>(v);
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                float w[16];
                tm_ld16(tt + COL_TW + 16 * hh, w);
                tm_wait_ld();
#pragma unroll
                for (int k = 1 + 8 * hh; k < 9 + 8 * hh && k < 16; k++) v[k] = mul(v[k], f2(w[2 * (k - 1 - 8 * hh)], w[2 * (k - 1 - 8 * hh) + 1]));
            }
            {
                const int n1 = s & 15, n2i = s >> 4;
#pragma unroll
                for (int k1 = 0; k1 < 16; k1++) X1[x1pos(n1, k1, n2i)] = v[k1];
            }
            gsync();
            // the staging buffer is free: stage the group's next forward job
            {
                const int q = next_fwd(r);
                if (q >= 0) issue_stage(q);
            }
            // ---------------- S2: DFT16 over n2, twiddle W_256^(n1 k2)
            {
                const int n1 = s >> 4, k1 = s & 15;
#pragma unroll
                for (int n = 0; n < 16; n++) v[n] = X1[x1pos(n1, k1, n)];
                dft16<false>(v);
#pragma unroll
                for (int k = 1; k < 16; k++) v[k] = mul(v[k], tw2[k * 16 + n1]);
#pragma unroll
                for (int k2 = 0; k2 < 16; k2++) X2[x2pos(k1 + 16 * k2, n1)] = v[k2];
            }
            gsync();
            // ---------------- S3: DFT16 over n1 -> Z[c + 256 k3]
#pragma unroll
            for (int n = 0; n < 16; n++) v[n] = X2[x2pos(c, n)];
            dft16<false>(v);
            // ---------------- separation: 2 F0[k] = Z[k] + conj Z[N-k], 2 F1[k] = -i (Z[k] - conj Z[N-k])
            float2 zp[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                zp[7 - q].x = __shfl_xor_sync(0xffffffffu, v[8 + q].x, 1);
                zp[7 - q].y = __shfl_xor_sync(0xffffffffu, v[8 + q].y, 1);
            }
            if (special) {
                if (c == 0) {
                    zp[0] = v[0];
#pragma unroll
                    for (int q = 1; q < 8; q++) zp[q] = v[16 - q];
                } else {
#pragma unroll
                    for (int q = 0; q < 8; q++) zp[q] = v[15 - q];
                }
            }
            float o[32];                         // mode q: 2F0 (re, im), 2F1 (re, im)
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const float2 z = v[q], w = zp[q];
                o[4 * q] = z.x + w.x;
                o[4 * q + 1] = z.y - w.y;
                o[4 * q + 2] = z.y + w.y;
                o[4 * q + 3] = w.x - z.x;
            }
            if (special && c == 0) {             // pack mode 0 (DC) and the Nyquist mode (both real)
                const float2 zn = v[8];
                o[1] = 2.f * zn.x;
                o[3] = 2.f * zn.y;
            }
            // ---------------- epilogue
            if (job == PJ_A || job == PJ_B || job == PJ_P1 || job == PJ_P2) {
                const int kind = (job == PJ_A) ? 0 : (job == PJ_B || job == PJ_P1) ? 1 : 2;
                const uint32_t col = slot_col(kind, job == PJ_P1 || job == PJ_P2 ? -1 : rr);
                tm_st16_at<0>(tt + col, o);
                tm_st16_at<16>(tt + col + 16, o);
            } else if (job == PJ_C) {
                // B2' = B2 + S E3;  B3' = B3 + a2 (E1(p+1) - E1(p)) - S E2   (two modes per chunk)
                const float sNx = symN->x;
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    float ea[8], e1n[8], e1[8], sy[8];
                    tm_ld8(tt + slot_col(0, rr) + 8 * h, ea);
                    tm_ld8(tt + slot_col(1, rr) + 8 * h, e1n);
                    tm_ld8(tt + slot_col(1, rr - 1) + 8 * h, e1);
                    tm_ld8(tt + COL_SYM + 8 * h, sy);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 2; i++) {
                        float* ob = o + 8 * h + 4 * i;
                        const float sx = sy[4 * i], syy = sy[4 * i + 1];
                        const float e2x = ea[4 * i], e2y = ea[4 * i + 1], e3x = ea[4 * i + 2], e3y = ea[4 * i + 3];
                        const float d1x = e1n[4 * i] - e1[4 * i], d1y = e1n[4 * i + 1] - e1[4 * i + 1];
                        float b2x = ob[0] + (sx * e3x - syy * e3y), b2y = ob[1] + (sx * e3y + syy * e3x);
                        float b3x = ob[2] + a2 * d1x - (sx * e2x - syy * e2y);
                        float b3y = ob[3] + a2 * d1y - (sx * e2y + syy * e2x);
                        if (h == 0 && i == 0 && special && c == 0) {   // DC (S = 0) and Nyquist (S real)
                            b2y = ob[1] + sNx * e3y;
                            b3y = ob[3] + a2 * d1y - sNx * e2y;
                        }
                        ob[0] = b2x; ob[1] = b2y; ob[2] = b3x; ob[3] = b3y;
                    }
                    float t8[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) t8[q] = o[8 * h + q];
                    tm_st8(tt + slot_col(2, rr) + 8 * h, t8);
                }
            } else {                              // PJ_D
                // E2' = E2 + conj(S) B3' - cj j2;  E3' = E3 - conj(S) B2' - cj j3      (into EA(p))
                // E1'(p) = E1(p) + a2 (B3'(p) - B3'(p-1)) - cj1 j1                      (into EB(p).f1)
                const float4 sN = *symN;
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    float ea[8], bc[8], sy[8];
                    tm_ld8(tt + slot_col(0, rr) + 8 * h, ea);
                    tm_ld8(tt + slot_col(2, rr) + 8 * h, bc);
                    tm_ld8(tt + COL_SYM + 8 * h, sy);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 2; i++) {
                        float* ob = o + 8 * h + 4 * i;
                        const float sx = sy[4 * i], syy = sy[4 * i + 1], cj = sy[4 * i + 3];
                        const float b2x = bc[4 * i], b2y = bc[4 * i + 1], b3x = bc[4 * i + 2], b3y = bc[4 * i + 3];
                        // conj(S) b = (sx bx + sy by, sx by - sy bx)
                        float e2x = ea[4 * i] + (sx * b3x + syy * b3y) - cj * ob[0];
                        float e2y = ea[4 * i + 1] + (sx * b3y - syy * b3x) - cj * ob[1];
                        float e3x = ea[4 * i + 2] - (sx * b2x + syy * b2y) - cj * ob[2];
                        float e3y = ea[4 * i + 3] - (sx * b2y - syy * b2x) - cj * ob[3];
                        if (h == 0 && i == 0 && special && c == 0) {   // Nyquist halves: S real, its own cj
                            e2y = ea[1] + sN.x * b3y - sN.w * ob[1];
                            e3y = ea[3] - sN.x * b2y - sN.w * ob[3];
                        }
                        ob[0] = e2x; ob[1] = e2y; ob[2] = e3x; ob[3] = e3y;
                    }
                    {
                        float t8[8];
#pragma unroll
                        for (int q = 0; q < 8; q++) t8[q] = o[8 * h + q];
                        tm_st8(tt + slot_col(0, rr) + 8 * h, t8);
                    }
                }
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    // EB(p) = (E1(p+1), j1(p)): j1 is replaced by E1'(p), E1(p+1) kept
                    float e1[8], bc[8], bp[8], eb[8], sy[8];
                    tm_ld8(tt + slot_col(1, rr - 1) + 8 * h, e1);
                    tm_ld8(tt + slot_col(2, rr) + 8 * h, bc);
                    tm_ld8(tt + slot_col(2, rr - 1) + 8 * h, bp);
                    tm_ld8(tt + slot_col(1, rr) + 8 * h, eb);
                    tm_ld8(tt + COL_SYM + 8 * h, sy);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 2; i++) {
                        const float cj1 = sy[4 * i + 2];
                        float e1x = e1[4 * i] + a2 * (bc[4 * i + 2] - bp[4 * i + 2]) - cj1 * eb[4 * i + 2];
                        float e1y = e1[4 * i + 1] + a2 * (bc[4 * i + 3] - bp[4 * i + 3]) - cj1 * eb[4 * i + 3];
                        if (h == 0 && i == 0 && special && c == 0) e1y = e1[1] + a2 * (bc[3] - bp[3]) - sN.z * eb[3];
                        eb[4 * i + 2] = e1x;
                        eb[4 * i + 3] = e1y;
                    }
                    tm_st8(tt + slot_col(1, rr) + 8 * h, eb);
                }
            }
            tm_wait_st();
        } else if (job == PJ_P3) {
            // B3'(p0-1) = B3 + a2 (E1(p0) - E1(p0-1)) - S E2 from BC(p0-1) = (E2, B3) and EB(p0-1) = (E1(p0), E1(p0-1))
            const float4 sN = *symN;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                float bc[16], eb[16], sy[16];
                tm_ld16(tt + slot_col(2, -1) + 16 * h, bc);
                tm_ld16(tt + slot_col(1, -1) + 16 * h, eb);
                tm_ld16(tt + COL_SYM + 16 * h, sy);
                tm_wait_ld();
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float sx = sy[4 * i], syy = sy[4 * i + 1];
                    const float e2x = bc[4 * i], e2y = bc[4 * i + 1];
                    const float d1x = eb[4 * i] - eb[4 * i + 2], d1y = eb[4 * i + 1] - eb[4 * i + 3];
                    float b3x = bc[4 * i + 2] + a2 * d1x - (sx * e2x - syy * e2y);
                    float b3y = bc[4 * i + 3] + a2 * d1y - (sx * e2y + syy * e2x);
                    if (h == 0 && i == 0 && special && c == 0) b3y = bc[3] + a2 * d1y - sN.x * e2y;
                    bc[4 * i + 2] = b3x;
                    bc[4 * i + 3] = b3y;
                }
                tm_st16(tt + slot_col(2, -1) + 16 * h, bc);
            }
            tm_wait_st();
            // B1'(p0-1) = B1(p0-1) - a2 (E3(p0) - E3(p0-1)) into shared memory
            const float* b1 = a.B[0] + (size_t)rowp(-1) * N;
            const float* e3a = a.E[2] + (size_t)rowp(0) * N;
            const float* e3b = a.E[2] + (size_t)rowp(-1) * N;
            for (int i = s; i < N; i += T) b1s[i] = b1[i] - a2 * (e3a[i] - e3b[i]);
        } else if (job == PJ_E || job == PJ_F || job == PJ_G) {
            // ---------------- inverse: slot -> merge -> S3, S2, S1 inverse -> two rows
            float x[32];
            const uint32_t col = (job == PJ_E) ? slot_col(0, rr) : (job == PJ_F) ? slot_col(2, rr) : slot_col(1, rr);
                if (job == PJ_G && rr == H - 1) {
                // the last row's B1'(p) = B1(p) - a2 (E3(p1) - E3(p)): E3(p1) from the copy the next
                // strip published, B1'(p-1) kept by the row's A job
                const int p = rowp(rr);
                const float* b1 = a.B[0] + (size_t)p * N;
                const float* e3 = a.E[2] + (size_t)p * N;
                const float* e3n = a.halo + ((size_t)next * 7 + 1) * N;
                float bb[16], en[16];
#pragma unroll
                for (int n = 0; n < 16; n++) { bb[n] = fmaf(a2, e3[s + 256 * n], b1[s + 256 * n]); en[n] = __ldcg(e3n + s + 256 * n); }
                float* dsc = P.scratch + ((size_t)strip * 2 + (rr & 1)) * N;
                float* b1o = a.B[0] + (size_t)p * N;
#pragma unroll
                for (int n = 0; n < 16; n++) {
                    const float b1n = bb[n] - a2 * en[n];
                    __stcg(dsc + s + 256 * n, a2 * (b1n - b1s[s + 256 * n]));
                    stg_stream1(b1o + s + 256 * n, b1n);
                }
            }
            tm_ld16_at<0>(tt + col, x);
            tm_ld16_at<16>(tt + col + 16, x);
            tm_wait_ld();
            // merge: Z[c + 256 q] = 2F0 + i 2F1 (own modes, q < 8); for q >= 8 the conjugate
            // combination of the partner column's mode 15 - q (or of own modes for 0 and 128)
            float2 v[16], wq[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const float f0x = x[4 * q], f0y = x[4 * q + 1], f1x = x[4 * q + 2], f1y = x[4 * q + 3];
                v[q] = f2(f0x - f1y, f0y + f1x);
                wq[q] = f2(f0x + f1y, f1x - f0y);
            }
            float2 pw[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                pw[q].x = __shfl_xor_sync(0xffffffffu, wq[q].x, 1);
                pw[q].y = __shfl_xor_sync(0xffffffffu, wq[q].y, 1);
            }
#pragma unroll
            for (int q = 8; q < 16; q++) v[q] = pw[15 - q];
            if (special) {
                if (c == 0) {
                    // packed mode 0: (2F0(0), 2F0(N)) and (2F1(0), 2F1(N)) are real
                    v[0] = f2(x[0], x[2]);
                    v[8] = f2(x[1], x[3]);
#pragma unroll
                    for (int q = 9; q < 16; q++) v[q] = wq[16 - q];
                } else {
#pragma unroll
                    for (int q = 8; q < 16; q++) v[q] = wq[15 - q];
                }
            }
            // ---------------- S3 inverse: DFT16 over k3 -> n1
            dft16<true>(v);
#pragma unroll
            for (int n = 0; n < 16; n++) X2[x2pos(c, n)] = v[n];
            gsync();
            // ---------------- S2 inverse: conj twiddle W_256^(n1 k2), DFT16 over k2 -> n2
            {
                const int n1 = s >> 4, k1 = s & 15;
#pragma unroll
                for (int k = 0; k < 16; k++) v[k] = X2[x2pos(k1 + 16 * k, n1)];
#pragma unroll
                for (int k = 1; k < 16; k++) v[k] = mulc(v[k], tw2[k * 16 + n1]);
                dft16<true>(v);
#pragma unroll
                for (int n = 0; n < 16; n++) X1[x1pos(n1, k1, n)] = v[n];
            }
            gsync();
            // ---------------- S1 inverse: conj twiddle W_4096^(s k1), DFT16 over k1 -> n3
            float corr[16];
            if (job == PJ_E) {                   // a2 (B1'(p) - B1'(p-1)), loaded while S1 runs
                const float* dsc = P.scratch + ((size_t)strip * 2 + (rr & 1)) * N;
#pragma unroll
                for (int n = 0; n < 16; n++) corr[n] = __ldcg(dsc + s + 256 * n);
            }
            {
                const int n1 = s & 15, n2i = s >> 4;
#pragma unroll
                for (int k = 0; k < 16; k++) v[k] = X1[x1pos(n1, k, n2i)];
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    float w[16];
                    tm_ld16(tt + COL_TW + 16 * hh, w);
                    tm_wait_ld();
#pragma unroll
                    for (int k = 1 + 8 * hh; k < 9 + 8 * hh && k < 16; k++) v[k] = mulc(v[k], f2(w[2 * (k - 1 - 8 * hh)], w[2 * (k - 1 - 8 * hh) + 1]));
                }
            }
            dft16<true>(v);
            const int p = rowp(rr);
            if (job == PJ_E) {
                float* d2 = a.E[1] + (size_t)p * N;
                float* d3 = a.E[2] + (size_t)p * N;
#pragma unroll
                for (int n = 0; n < 16; n++) {
                    stg_stream1(d2 + s + 256 * n, v[n].x * INV2N);
                    stg_stream1(d3 + s + 256 * n, v[n].y * INV2N - corr[n]);
                }
            } else if (job == PJ_F) {
                float* d2 = a.B[1] + (size_t)p * N;
                float* d3 = a.B[2] + (size_t)p * N;
#pragma unroll
                for (int n = 0; n < 16; n++) {
                    stg_stream1(d2 + s + 256 * n, v[n].x * INV2N);
                    stg_stream1(d3 + s + 256 * n, v[n].y * INV2N);
                }
            } else {                              // G: EB(p) = (E1(p+1), E1'(p)): E1' is the second row
                float* d1 = a.E[0] + (size_t)p * N;
#pragma unroll
                for (int n = 0; n < 16; n++) stg_stream1(d1 + s + 256 * n, v[n].y * INV2N);
            }
        }
        tm_wait_st();
        if (sy & PS_END) {
            tm_fence_before();
            gsync();
            if (s == 0) {
                __threadfence_block();
                done[g * MAXR + r] = 1;
                if (fl & (PF_SET_PUB | PF_SET_READ)) {
                    __threadfence();
                    if (fl & PF_SET_PUB) st_release(P.flags + 2 * strip, P.epoch);
                    if (fl & PF_SET_READ) st_release(P.flags + 2 * strip + 1, P.epoch);
                }
            }
        }
    }
    // a bulk load still in flight (only after an aborted wait) must land before the CTA exits
    if (pending && s == 0) {
        const long long t0 = clock64();
        while (!mbar_try_wait(bar, nld & 1) && clock64() - t0 < kWaitCycles) {}
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(tbase, TMEM_COLS);
}

// ------------------------------------------------------------------ host: the schedule of a strip
// Jobs of a strip of H rows (rows rr = 0..H-1 relative to p0; rr = -1 the row before) and the
// jobs each one waits for: data flow through the TMEM slots, the reuse of each slot by the row
// two below, the B1' and E3 rows in shared memory and the scratch rows, and the global rows each
// job overwrites.  List scheduling on two groups gives each group its sequence of jobs (entry q
// of the table is the q-th job of each group); at run time a job waits only for the jobs of the
// other group it depends on, through per-job done flags.
static std::vector<PJob> pair_schedule(int H) {
    struct J { int kind, row; };
    std::vector<J> jobs = {{PJ_P1, -1}, {PJ_P2, -1}, {PJ_P3, -1}};
    for (int r = 0; r < H; r++)
        for (int k : {PJ_A, PJ_B, PJ_C, PJ_D, PJ_F, PJ_G, PJ_E}) jobs.push_back({k, r});
    auto id = [&](int kind, int row) -> int {
        for (size_t i = 0; i < jobs.size(); i++) if (jobs[i].kind == kind && jobs[i].row == row) return (int)i;
        return -1;
    };
    std::vector<std::vector<int>> dep(jobs.size());
    auto add = [&](int i, int kind, int row) { const int j = id(kind, row); if (j >= 0) dep[i].push_back(j); };
    const int last = H - 1;
    for (size_t i = 0; i < jobs.size(); i++) {
        const int k = jobs[i].kind, r = jobs[i].row;
        switch (k) {
        case PJ_P3: add(i, PJ_P1, -1); add(i, PJ_P2, -1); break;
        case PJ_A:                       // EA slot reuse; the B1' row in shared memory; scratch row reuse
            add(i, PJ_E, r - 2); add(i, PJ_E, r - 3); add(i, PJ_A, r - 1);
            if (r == 0) add(i, PJ_P1, -1);
            if (r == 1) add(i, PJ_P3, -1);
            break;
        case PJ_B: add(i, PJ_D, r - 1); add(i, PJ_G, r - 2); break;
        case PJ_C:
            add(i, PJ_A, r); add(i, PJ_B, r); add(i, PJ_D, r - 1); add(i, PJ_F, r - 2);
            if (r == 0) add(i, PJ_P1, -1); else add(i, PJ_B, r - 1);
            break;
        case PJ_D: add(i, PJ_C, r); if (r == 0) add(i, PJ_P3, -1); else add(i, PJ_C, r - 1); break;
        case PJ_E: add(i, PJ_D, r); if (r < last) add(i, PJ_A, r + 1); else add(i, PJ_G, r); break;
        case PJ_F: add(i, PJ_C, r); break;
        case PJ_G: add(i, PJ_D, r); break;
        }
    }
    // event-driven list scheduling: the group that frees first takes, of the jobs whose
    // dependencies will have finished by then, the first in priority order (else the one that
    // becomes ready first), with estimated costs in units of a plain transform pair
    auto cost = [](int k) {
        switch (k) {
        case PJ_C: return 1.15;
        case PJ_D: return 1.35;
        case PJ_A: return 1.1;
        case PJ_P3: return 0.3;
        default: return 1.0;
        }
    };
    // priority: the longest chain of costs from a job to the end of the strip (critical path first)
    std::vector<double> level(jobs.size(), 0.0);
    for (int it = 0; it < (int)jobs.size(); it++)
        for (size_t i = 0; i < jobs.size(); i++)
            for (int d : dep[i]) level[d] = std::max(level[d], level[i] + cost(jobs[i].kind));
    std::vector<int> round_of(jobs.size(), -1), group_of(jobs.size(), -1);
    std::vector<double> fin(jobs.size(), 0.0);
    std::vector<int> seq[2];
    double free_at[2] = {0.0, 0.0};
    for (size_t n = 0; n < jobs.size(); n++) {
        const int g = free_at[0] <= free_at[1] ? 0 : 1;
        int best = -1, best_now = -1;
        double best_ready = 1e30;
        for (size_t i = 0; i < jobs.size(); i++) {
            if (group_of[i] >= 0) continue;
            bool sched = true;
            double ready = 0.0;
            for (int d : dep[i]) {
                if (group_of[d] < 0) { sched = false; break; }
                ready = std::max(ready, fin[d]);
            }
            if (!sched) continue;
            if (ready <= free_at[g]) {
                if (best_now < 0 || level[i] > level[best_now]) best_now = (int)i;
            } else if (ready < best_ready || (ready == best_ready && level[i] > level[best])) {
                best = (int)i;
                best_ready = ready;
            }
        }
        if (best_now >= 0) { best = best_now; best_ready = free_at[g]; }
        const double start = std::max(free_at[g], best_ready);
        fin[best] = start + cost(jobs[best].kind);
        free_at[g] = fin[best];
        group_of[best] = g;
        round_of[best] = (int)seq[g].size();
        seq[g].push_back(best);
    }
    const size_t R = std::max(seq[0].size(), seq[1].size());
    std::vector<PJob> out(2 * R);        // [group][position]
    for (auto& e : out) {
        e = PJob{};
        e.job = PJ_IDLE;
    }
    for (int g = 0; g < 2; g++)
        for (size_t q = 0; q < seq[g].size(); q++) {
            out[g * R + q].job = (int8_t)jobs[seq[g][q]].kind;
            out[g * R + q].row = (int8_t)jobs[seq[g][q]].row;
        }
    auto fwd = [](int k) { return k == PJ_A || k == PJ_B || k == PJ_C || k == PJ_D || k == PJ_P1 || k == PJ_P2; };
    auto inv = [](int k) { return k == PJ_E || k == PJ_F || k == PJ_G; };
    std::vector<bool> awaited(jobs.size(), false);
    for (size_t i = 0; i < jobs.size(); i++)
        for (int d : dep[i]) if (group_of[d] != group_of[i]) awaited[d] = true;
    for (size_t i = 0; i < jobs.size(); i++) {
        const int r = round_of[i], g = group_of[i];
        PJob& e = out[g * R + r];
        unsigned long long m = 0;
        for (int d : dep[i]) if (group_of[d] != g) m |= 1ull << round_of[d];
        e.dep = m;
        const int k = jobs[i].kind, row = jobs[i].row;
        int f = 0;
        // the next strip's published rows: read by B and G of the last row; the last row itself:
        // read by the next strip's prologue before E, F, G overwrite it
        if (row == last && (k == PJ_B || k == PJ_G)) f |= PF_WAIT_PUB;
        if (row == last && (k == PJ_E || k == PJ_F || k == PJ_G)) f |= PF_WAIT_READ;
        if (k == PJ_A && row == 0) f |= PF_SET_PUB;       // after P1 (a dependency) and A(0) published
        if (k == PJ_P3) f |= PF_SET_READ;
        e.flags = (uint8_t)f;
        // a barrier after the job: when the other group waits for it, when it sets a flag for the
        // neighbour strip, and when the group's next job would write an exchange buffer this one
        // may still be reading (a forward job ends reading X2, which an inverse writes first; an
        // inverse ends reading X1, which a forward writes first)
        const int nk = (r + 1 < (int)seq[g].size()) ? jobs[seq[g][r + 1]].kind : PJ_IDLE;
        const bool race = (fwd(k) && inv(nk)) || (inv(k) && fwd(nk));
        e.sync = (uint8_t)(((m != 0 || (f & (PF_WAIT_PUB | PF_WAIT_READ))) ? PS_START : 0) |
                           ((awaited[i] || (f & (PF_SET_PUB | PF_SET_READ)) || race) ? PS_END : 0));
    }
    return out;
}

size_t fused_pair_smem_bytes() { return (size_t)pq::SMEM; }

cudaError_t fused_pair_occupancy(int* occ) {
    cudaError_t e = func_attr_once((const void*)k_fused_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, pq::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_fused_pair, pq::NT, pq::SMEM);
    if (e == cudaSuccess && *occ > 1) *occ = 1;     // TMEM holds one CTA's slots per SM
    return e;
}

// per-grid state of the paired kernel: schedules for the grid's two strip heights, the
// W_4096 table, the scratch rows
struct PairPlan {
    int n2 = 0, ns = 0;           // the grid's rows and strips the plan was made for
    PJob* sched = nullptr;
    int nrounds[2] = {0, 0};
    int hs[2] = {0, 0};
    float2* tw = nullptr;
    float* scratch = nullptr;
};
static std::mutex g_pair_mu;
static std::map<const FusedPlan*, PairPlan> g_pair;

void fused_pair_release(const FusedPlan* P) {
    std::lock_guard<std::mutex> lk(g_pair_mu);
    auto it = g_pair.find(P);
    if (it == g_pair.end()) return;
    if (it->second.sched) cudaFree(it->second.sched);
    if (it->second.tw) cudaFree(it->second.tw);
    if (it->second.scratch) cudaFree(it->second.scratch);
    g_pair.erase(it);
}

static cudaError_t pair_plan(const FusedBatch& fb, const FusedPlan* FP, PairPlan** out) {
    std::unique_lock<std::mutex> lk(g_pair_mu);
    const int n2 = fb.inst[0].n2, ns = fb.n_strips;
    auto it = g_pair.find(FP);
    if (it != g_pair.end()) {
        if (it->second.n2 == n2 && it->second.ns == ns) { *out = &it->second; return cudaSuccess; }
        lk.unlock();
        fused_pair_release(FP);               // made for another strip count: rebuild
        lk.lock();
    }
    PairPlan pp;
    pp.n2 = n2;
    pp.ns = ns;
    // strip heights of fused_items: floor and ceil of n2 / ns
    pp.hs[0] = n2 / ns;
    pp.hs[1] = (n2 + ns - 1) / ns;
    std::vector<PJob> s0 = pair_schedule(pp.hs[0]), s1 = pair_schedule(pp.hs[1]);
    if ((int)s0.size() > 2 * pq::MAXR || (int)s1.size() > 2 * pq::MAXR) return cudaErrorInvalidValue;
    pp.nrounds[0] = (int)s0.size() / 2;
    pp.nrounds[1] = (int)s1.size() / 2;
    cudaError_t e = cudaMalloc(&pp.sched, sizeof(PJob) * (s0.size() + s1.size()));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(pp.sched, s0.data(), sizeof(PJob) * s0.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pp.sched + s0.size(), s1.data(), sizeof(PJob) * s1.size(), cudaMemcpyHostToDevice);
    std::vector<float2> tw(pq::N);
    for (int j = 0; j < pq::N; j++) {
        const double ang = -2.0 * 3.14159265358979323846 * j / pq::N;
        tw[j] = make_float2((float)cos(ang), (float)sin(ang));
    }
    if (e == cudaSuccess) e = cudaMalloc(&pp.tw, sizeof(float2) * pq::N);
    if (e == cudaSuccess) e = cudaMemcpy(pp.tw, tw.data(), sizeof(float2) * pq::N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&pp.scratch, sizeof(float) * 2 * (size_t)ns * pq::N);
    if (e != cudaSuccess) {
        if (pp.sched) cudaFree(pp.sched);
        if (pp.tw) cudaFree(pp.tw);
        if (pp.scratch) cudaFree(pp.scratch);
        return e;
    }
    g_pair[FP] = pp;
    *out = &g_pair[FP];
    return cudaSuccess;
}

bool fused_pair_applies(const FusedBatch& fb) {
    // strips of 2 to 8 rows (a group's job list for 8 rows has about 30 jobs, within MAXR)
    return fb.flags != nullptr && fb.inst[0].n2 >= 2 * fb.n_strips && fb.inst[0].n2 <= 8 * fb.n_strips &&
           fb.n_items == fb.n_strips;
}

cudaError_t fused_pair_launch(const FusedBatch& fb, const FusedPlan* FP, int grid, cudaStream_t s) {
    PairPlan* pp = nullptr;
    cudaError_t e = pair_plan(fb, FP, &pp);
    if (e != cudaSuccess) return e;
    PairArgs A;
    A.a = fb.inst[0];
    A.items = fb.items;
    A.sched[0] = pp->sched;
    A.sched[1] = pp->sched + 2 * pp->nrounds[0];
    A.nrounds[0] = pp->nrounds[0];
    A.nrounds[1] = pp->nrounds[1];
    A.hs[0] = pp->hs[0];
    A.hs[1] = pp->hs[1];
    A.tw = pp->tw;
    A.scratch = pp->scratch;
    A.flags = fb.flags;
    A.epoch = fb.epoch;
    A.n_strips = fb.n_strips;
    A.err = fb.err;
    e = func_attr_once((const void*)k_fused_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, pq::SMEM);
    if (e != cudaSuccess) return e;
    void* args[] = {&A};
    return cudaLaunchCooperativeKernel((const void*)k_fused_pair, dim3(grid), dim3(pq::NT), args, pq::SMEM, s);
}

}  // namespace hyb
