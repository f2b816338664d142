// tmt_body.cuh -- the n1 = 512, 1024, 2048 fused FP32 advance as a device function of one
// 384-thread team CTA, so that the kernel of fused_tmt.cu and the single-launch batched step
// (batch_step.cu) run the same code.
//
// Single-pass FP32 hybrid advance for n1 = 512, 1024 and 2048
// with the k1-space lines in tensor memory: the schedule, slots, epilogues and
// bulk-copy staging of the n1 = 4096 kernel (tm_body.cuh), re-laid for rows of
// 16 T points (T = 32, 64, 128 threads per group, 8 complex points a thread):
//
//   * a CTA is 12 warps (384 threads) in 128 / T teams; each team is three groups
//     of T threads (components 1, 2, 3 of E and B) and sweeps its own strip of x2
//     rows.  Group g of team tm is made of the warps 4 g + q whose TMEM lane
//     quarter q belongs to the team, so thread t of every group of a team sits in
//     the same TMEM lane and owns the same 8 modes: the per-mode updates are
//     lane-local tcgen05.ld / tcgen05.st, as in the n1 = 4096 kernel;
//   * 256 TMEM columns per CTA (10 slots of 16 words, symbols 32, twiddles 64),
//     two CTAs per SM: 24 warps per SM at every n1;
//   * the complex M = 8 T-point FFT of z[j] = x[2j] + i x[2j+1] is factored
//     8 x 8 x U x 4 (U = T / 32):
//       S1  thread t holds z[t + T n], 8-point DFT over n -> k1, twiddle W_M^{t k1};
//       S2  thread (t0, k1), t = t0 + T0 k1 (T0 = T / 8): 8-point DFT over t1 -> k2,
//           twiddle W_T^{t0 k2};
//       S3  (U > 1) t0 = u0 + 4 u1: U-point DFT over u1 -> k3, twiddle W_T0^{u0 k3}
//           (the warp of S2 threads (., k1) handles those k1, lanes (u0, k2));
//       S4  thread t owns columns c = k1 + 8 k2 + 64 k3 in {t, 2T - t} (t = 0:
//           {0, T}), 4-point DFT over u0 -> Z[c + 2T k4];
//     so Z[kappa] and Z[M - kappa] sit in one thread and the even/odd split of the
//     real transform is done in registers.  The inverse runs the stages transposed.
//   * shared memory per group: the staging row of the next forward transform and
//     three exchange buffers: A (S1 -> S2), Y (S2 -> S3, inside a warp), B (S3 -> S4);
//     the inverse uses A and B the other way round (S4 -> S3 in A, S2 -> S1 in B),
//     so that no transform's first write meets the last reads of the one before it.
// The exchange paddings and the column permutation of the S3 -> S4 exchange were chosen
// with a bank model of the accesses: every access is conflict-free except the S3 reads
// (T = 64) and half of the S4 reads of the second column, 2-way.
#pragma once
#include <math.h>

#include "fused_api.cuh"
#include "fused_dev.cuh"
#include "packed_dev.cuh"
#include "tm_dev.cuh"
#include "tm_sched.cuh"

namespace hyb {

template <int T>
struct Tmt {
    static constexpr int N = 16 * T, M = 8 * T, C = 2 * T, T0 = T / 8, U1 = T0 / 4;
    static constexpr int WPG = T / 32;                  // warps per group
    static constexpr int NTM = 128 / T;                 // teams per CTA
    static constexpr int NT = 384;
    static constexpr int P1 = (T == 32) ? 4 : (T == 64) ? 8 : 0;
    static constexpr int P2 = (T == 64) ? 1 : (T == 128) ? 4 : 0;
    static constexpr int P3 = (T == 32) ? 4 : 1;
    static constexpr int XR = T + P1, YR = T0 + P2, CR = C + P3;
    static constexpr int BUF = (8 * XR > 4 * CR ? 8 * XR : 4 * CR);
    static constexpr int YBUF = (U1 > 1) ? 64 * YR : 0;
    static constexpr int GS = ((M + 2 * BUF + YBUF + 1) / 2) * 2;   // float2 per group (16-byte multiple)
    static constexpr int NG = 3 * NTM;                              // groups per CTA
    static constexpr int OFF_SYMN = NG * GS * 8;                    // float4 per team
    static constexpr int OFF_BAR = OFF_SYMN + 16 * NTM;             // one mbarrier per group
    static constexpr int OFF_MISC = OFF_BAR + 8 * NG;               // TMEM base address, abort flags (per group)
    static constexpr int SMEM = OFF_MISC + 4 + 4 * NG;
    // inside the single-launch batched step: one mbarrier per team (the team barrier at T = 64) after them
    static constexpr int OFF_TBAR = (SMEM + 7) / 8 * 8;
    static constexpr int SMEM_MEGA = (OFF_TBAR + 8 * NTM + 127) / 128 * 128;
    // named barriers of a half: group barriers (groups of more than one warp), team barriers
    // (none at T = 64 inside the batched step, where they are mbarriers)
    static constexpr int NGB = (WPG > 1) ? 3 * NTM : 0;
    static constexpr uint32_t TMEM_COLS = 256;                      // slots 160, symbols 32, twiddles 64
    static constexpr int SYM_COL = 160, TW_COL = 192;
};

template <bool INV>
__device__ __forceinline__ void dft2x(float2& a, float2& b) {
    const float2 s = vadd(a, b), d = vsub(a, b);
    a = s;
    b = d;
}

// One team CTA of 384 threads sweeping the work items of its teams: vb NTM + tm, then steps of
// vg NTM.  tid is the thread's index in the 384, sm its dynamic shared memory.  Standalone (MEGA =
// false) it is a whole CTA and allocates its 256 TMEM columns; in the single-launch batched step
// it is half `half` of a 768-thread CTA whose TMEM columns tbase_in .. + 255 the caller allocated.
template <int T, bool MEGA>
__device__ __forceinline__ void tmt_body(const FusedBatch& fb, const int vb, const int vg, const int tid,
                                         unsigned char* sm, const int half, const uint32_t tbase_in) {
    using G = Tmt<T>;
    constexpr int N = G::N, M = G::M, C = G::C, T0 = G::T0, U1 = G::U1, NTM = G::NTM, WPG = G::WPG;
    constexpr int XR = G::XR, YR = G::YR, CR = G::CR;
    const int warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3;                      // TMEM lane quarter of this warp
    const int g = warp >> 2;                     // component (group) 0..2
    const int tm = q / WPG;                      // team
    const int t = (q % WPG) * 32 + lane;         // thread within the group
    const int gi = tm * 3 + g;                   // group index in the CTA
    float2* stg = reinterpret_cast<float2*>(sm) + (size_t)gi * G::GS;
    float2* bA = stg + M;
    float2* bB = bA + G::BUF;
    float2* bY = bB + G::BUF;
    float4* symN = reinterpret_cast<float4*>(sm + G::OFF_SYMN) + tm;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + G::OFF_BAR);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(sm + G::OFF_MISC);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + G::OFF_MISC + 4) + gi;
    const bool fm = fb.flags != nullptr;
    if (vb * NTM >= fb.n_items) return;
    constexpr bool TEAM_MB = MEGA && T == 64;
    constexpr int NTB = TEAM_MB ? 0 : NTM;
    const int bar0 = 1 + half * (G::NGB + NTB);       // first named barrier of this half
    // all 384 threads: the CTA, or this half of it (named barrier 13 + half)
    auto cta_bar = [&]() {
        if constexpr (MEGA) asm volatile("bar.sync %0, 384;" :: "r"(13 + half) : "memory");
        else __syncthreads();
    };

    // ---- one-time set-up: TMEM, barriers, twiddles
    if (!MEGA && warp == 0) {
        tm_alloc(smem_addr(s_taddr), G::TMEM_COLS);
        tm_relinquish();
    }
    if (tid < G::NG) {
        mbar_init(smem_addr(bars + tid), 1);
        reinterpret_cast<volatile int*>(sm + G::OFF_MISC + 4)[tid] = 0;
    }
    uint64_t* tbars = reinterpret_cast<uint64_t*>(sm + G::OFF_TBAR);
    if constexpr (TEAM_MB) {
        if (tid < NTM) mbar_init(smem_addr(tbars + tid), 3 * T);
    }
    if (tid == 0) mbar_fence_init();
    const FusedInst& i0 = fb.inst[fb.items[vb * NTM].x];
    tm_fence_before();
    cta_bar();
    tm_fence_after();
    const uint32_t tbase = MEGA ? tbase_in : *s_taddr;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    const uint32_t tw = tbase + lanes;                               // slot s, chunk c at tw + 16 s + 8 c
    const uint32_t ts = tbase + lanes + (uint32_t)G::SYM_COL;        // symbols of this thread's modes
    const uint32_t twc = tbase + lanes + (uint32_t)G::TW_COL;        // stage and split twiddles

    // modes owned by this thread
    const int cA = t, cB = (t == 0) ? C / 2 : C - t;
    auto kap = [&](int e) { return (e & 1) ? cB + C * (3 - (e >> 1)) : cA + C * (e >> 1); };
    // stage thread maps
    const int s2_t0 = t % T0, s2_k1 = t / T0;
    const int s3_u0 = lane & 3, s3_k2 = (lane >> 2) & 7, s3_w = t >> 5;
    constexpr int NK1 = (U1 > 1) ? 32 / T0 : 1;                     // k1 values per warp in S3
    constexpr float inv2M = 0.5f / (float)M;
    // position of (u0, column c) in the S3 -> S4 exchange: for U > 1 bit 2 of c is flipped by its bits
    // 4 and 5 (a permutation of the columns), which keeps the S3 writes free of bank conflicts
    auto x3 = [&](int u0, int c) {
        if constexpr (U1 > 1) c ^= (((c >> 4) ^ (c >> 5)) & 1) << 2;
        return u0 * CR + c;
    };

    // this thread's twiddles into TMEM (written by group 0 of each team)
    if (g == 0) {
        float r[16];
        auto put = [&](int step, int i, uint32_t col) {      // W_M^{step i k}, k = 1..7
#pragma unroll
            for (int k = 1; k < 8; k++) {
                const float2 w = i0.twM[(step * i * k) & (M - 1)];
                r[2 * k - 2] = w.x;
                r[2 * k - 1] = w.y;
            }
            r[14] = 0.f;
            r[15] = 0.f;
            tm_st16(twc + col, r);
        };
        put(1, t, 0);                 // S1: W_M^{t k}
        put(8, s2_t0, 16);            // S2: W_T^{t0 k}
        put(64, s3_u0, 32);           // S3: W_T0^{u0 k}
        const float2 wA = i0.twC[t];  // W_N^{cA}
        float qv[8];
#pragma unroll
        for (int k4 = 0; k4 < 4; k4++) {
            const float2 w = mul(wA, wr(8, k4));
            qv[2 * k4] = w.x;
            qv[2 * k4 + 1] = w.y;
        }
        tm_st8(twc + 48, qv);
        tm_wait_st();
    }
    tm_fence_before();
    cta_bar();
    tm_fence_after();

    const uint32_t bar = smem_addr(bars + gi);
    const uint32_t stg_s = smem_addr(stg);
    uint32_t nld = 0;          // bulk loads of this group consumed so far (mbarrier phase)
    int cur_inst = -1;
    bool pending = false;      // a bulk load issued and not yet consumed

    auto gsync = [&]() {
        if (WPG == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;" :: "r"(bar0 + gi), "r"(T) : "memory");
    };
    const int team_bar = bar0 + G::NGB + tm;
    const uint32_t tbar = smem_addr(tbars + tm);
    uint32_t tph = 0;          // phase of the team mbarrier (TEAM_MB)
    auto team_sync = [&]() {
        tm_fence_before();
        if constexpr (TEAM_MB) {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tbar) : "memory");
            mbar_wait(tbar, tph, fb.err, s_abort);
            tph ^= 1;
        } else {
            asm volatile("bar.sync %0, %1;" :: "r"(team_bar), "r"(3 * T) : "memory");
        }
        tm_fence_after();
    };
    const bool leader = g == 0 && t == 0;

  for (int item = vb * NTM + tm; item < fb.n_items; item += vg * NTM) {
    const int4 it = fb.items[item];
    const FusedInst& a = fb.inst[it.x];
    const int strip = it.y, p0 = it.z, p1 = it.w;
    const int H = p1 - p0;
    const int nrounds = 3 + 5 * H;
    const float a2 = a.a2;
    const int next = fm ? (strip + 1) % fb.n_strips : 0;
    const int ri_wait_halo = 3 + 5 * (H - 1);
    const int ri_wait_read = 3 + 5 * (H - 1) + 3;
    auto sync_after = [&](int ri) {
        if (ri < 3) return ri >= 1 || fm;
        const int r = (ri - 3) % 5;
        return r == 0 || r == 1;
    };
    if (it.x != cur_inst) {
        team_sync();
        if (g == 0) {
            float r[16];
#pragma unroll
            for (int e = 0; e < 8; e++) { const float4 qs = a.sym[kap(e)]; r[2 * e] = qs.x; r[2 * e + 1] = qs.y; }
            tm_st16(ts, r);
#pragma unroll
            for (int e = 0; e < 8; e++) { const float4 qs = a.sym[kap(e)]; r[e] = qs.z; r[8 + e] = qs.w; }
            tm_st16(ts + 16, r);
            tm_wait_st();
        }
        if (leader) *symN = a.sym[M];
        team_sync();
        cur_inst = it.x;
    }
    int fidx = 0;
    bool ndirect = false;
    const float* nsrc = tm_src(a, N, strip, p0, p1, g, 0, fm, next, &ndirect);
    pending = nsrc != nullptr && !ndirect;
    if (pending && t == 0) {
        mbar_expect_tx(bar, 4 * N);
        bulk_load(stg_s, nsrc, 4 * N, bar);
    }

    for (int ri = 0; ri < nrounds; ri++) {
        if (fm && (ri == ri_wait_halo || ri == ri_wait_read)) {
            if (leader) wait_flag(fb.flags + 2 * next + (ri == ri_wait_read ? 1 : 0), fb.epoch, fb.err);
            team_sync();
        }
        const Job j = tm_job(a, N, p0, p1, ri, g);
        if (j.kind == J_FWD) {
            // ---------------- S1: 8-point DFT of z[t + T n]
            float2 v[8];
            if (ndirect) {
                const float2* s = reinterpret_cast<const float2*>(nsrc);
#pragma unroll
                for (int n = 0; n < 8; n++) v[n] = ldg_stream(s + t + T * n);
            } else {
                mbar_wait(bar, nld & 1, fb.err, s_abort);
                nld++;
                pending = false;
#pragma unroll
                for (int n = 0; n < 8; n++) v[n] = stg[t + T * n];
            }
            if (fm && ri == 0 && g != 1) {
                // publish E1 (g = 0) or E3 (g = 2) of the strip's first row for the previous strip
                float2* h = reinterpret_cast<float2*>(const_cast<float*>(a.halo) + ((size_t)strip * 7 + (g == 0 ? 0 : 1)) * N);
#pragma unroll
                for (int n = 0; n < 8; n++) h[t + T * n] = v[n];
            }
            dft8x<false>(v);
            {
                float2 w[8];
                tw_tmem(twc, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mul(v[k], w[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; k++) bA[k * XR + t] = v[k];
            gsync();
            fidx++;
            // the group's staging row is free: start the next forward's row
            nsrc = tm_src(a, N, strip, p0, p1, g, fidx, fm, next, &ndirect);
            pending = nsrc != nullptr && !ndirect;
            if (pending && t == 0) {
                fence_proxy_async_smem();
                mbar_expect_tx(bar, 4 * N);
                bulk_load(stg_s, nsrc, 4 * N, bar);
            }
            // ---------------- S2: over t1 -> k2
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = bA[s2_k1 * XR + s2_t0 + T0 * n];
            dft8x<false>(v);
            {
                float2 w[8];
                tw_tmem(twc + 16, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mul(v[k], w[k]);
            }
            if constexpr (U1 == 1) {
#pragma unroll
                for (int k = 0; k < 8; k++) bB[x3(s2_t0, s2_k1 + 8 * k)] = v[k];
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++) bY[(s2_k1 * 8 + k) * YR + s2_t0] = v[k];
                __syncwarp();
                // ---------------- S3: over u1 -> k3 for the k1 of this warp, lanes (u0, k2)
                float2 w3[8];
                tw_tmem(twc + 32, w3);
#pragma unroll
                for (int ci = 0; ci < NK1; ci++) {
                    const int k1 = s3_w * NK1 + ci;
                    float2 u[U1];
#pragma unroll
                    for (int u1 = 0; u1 < U1; u1++) u[u1] = bY[(k1 * 8 + s3_k2) * YR + s3_u0 + 4 * u1];
                    if constexpr (U1 == 4) dft4x<false>(u[0], u[1], u[2], u[3]);
                    else dft2x<false>(u[0], u[1]);
#pragma unroll
                    for (int k3 = 0; k3 < U1; k3++)
                        bB[x3(s3_u0, k1 + 8 * s3_k2 + 64 * k3)] = (k3 == 0) ? u[0] : mul(u[k3], w3[k3]);
                }
            }
            gsync();
            // ---------------- S4: columns cA, cB, 4-point DFT over u0
            float2 A4[4], B4[4];
#pragma unroll
            for (int u = 0; u < 4; u++) { A4[u] = bB[x3(u, cA)]; B4[u] = bB[x3(u, cB)]; }
            dft4x<false>(A4[0], A4[1], A4[2], A4[3]);
            dft4x<false>(B4[0], B4[1], B4[2], B4[3]);
            // even/odd split into the real-input coefficients of this thread's modes
            float2 x[8];
            {
                float ws[8];
                tm_ld8(twc + 48, ws);
                tm_wait_ld();
#pragma unroll
                for (int k4 = 0; k4 < 4; k4++) split_fwd(A4[k4], B4[3 - k4], f2(ws[2 * k4], ws[2 * k4 + 1]), x[2 * k4], x[2 * k4 + 1]);
            }
            if (t == 0) {
                // columns 0 and T pair with themselves: Z[0] gives (X_0, X_M), Z[2T] with Z[6T],
                // Z[4T] with itself, Z[T] with Z[7T], Z[3T] with Z[5T]
                x[0] = f2(A4[0].x + A4[0].y, A4[0].x - A4[0].y);
                split_fwd(A4[1], A4[3], wconst<8, 1, false>(), x[2], x[6]);
                float2 dummy;
                split_fwd(A4[2], A4[2], wconst<4, 1, false>(), x[4], dummy);
                split_fwd(B4[0], B4[3], wconst<16, 1, false>(), x[7], x[1]);
                split_fwd(B4[1], B4[2], wconst<16, 3, false>(), x[5], x[3]);
            }
            // ---------------- epilogue: per-mode updates, two chunks of four modes
            tm_epilogue(j, x, tw, ts, symN, a2, t == 0);
        } else if (j.kind == J_INV) {
            // ---------------- slot -> inverse split -> inverse 4-point DFT over k4 (into A)
            float2 x[8];
            {
                float r0[8], r1[8], ws[8];
                tm_ld8(tw + (uint32_t)(16 * j.slot), r0);
                tm_ld8(tw + (uint32_t)(16 * j.slot + 8), r1);
                tm_ld8(twc + 48, ws);
                tm_wait_ld();
#pragma unroll
                for (int i = 0; i < 4; i++) { x[i] = f2(r0[2 * i], r0[2 * i + 1]); x[4 + i] = f2(r1[2 * i], r1[2 * i + 1]); }
                float2 A4[4], B4[4];
#pragma unroll
                for (int k4 = 0; k4 < 4; k4++)
                    split_inv(x[2 * k4], x[2 * k4 + 1], f2(ws[2 * k4], ws[2 * k4 + 1]), inv2M, A4[k4], B4[3 - k4]);
                if (t == 0) {
                    A4[0] = f2((x[0].x + x[0].y) * inv2M, (x[0].x - x[0].y) * inv2M);
                    split_inv(x[2], x[6], wconst<8, 1, false>(), inv2M, A4[1], A4[3]);
                    float2 dummy;
                    split_inv(x[4], x[4], wconst<4, 1, false>(), inv2M, A4[2], dummy);
                    split_inv(x[7], x[1], wconst<16, 1, false>(), inv2M, B4[0], B4[3]);
                    split_inv(x[5], x[3], wconst<16, 3, false>(), inv2M, B4[1], B4[2]);
                }
                dft4x<true>(A4[0], A4[1], A4[2], A4[3]);
                dft4x<true>(B4[0], B4[1], B4[2], B4[3]);
#pragma unroll
                for (int u = 0; u < 4; u++) { bA[x3(u, cA)] = A4[u]; bA[x3(u, cB)] = B4[u]; }
            }
            gsync();
            float2 v[8];
            if constexpr (U1 == 1) {
#pragma unroll
                for (int k = 0; k < 8; k++) v[k] = bA[x3(s2_t0, s2_k1 + 8 * k)];
            } else {
                // ---------------- S3 inverse: twiddle, inverse U-point DFT over k3 -> u1 (into Y)
                float2 w3[8];
                tw_tmem(twc + 32, w3);
#pragma unroll
                for (int ci = 0; ci < NK1; ci++) {
                    const int k1 = s3_w * NK1 + ci;
                    float2 u[U1];
#pragma unroll
                    for (int k3 = 0; k3 < U1; k3++) {
                        const float2 val = bA[x3(s3_u0, k1 + 8 * s3_k2 + 64 * k3)];
                        u[k3] = (k3 == 0) ? val : mulc(val, w3[k3]);
                    }
                    if constexpr (U1 == 4) dft4x<true>(u[0], u[1], u[2], u[3]);
                    else dft2x<true>(u[0], u[1]);
#pragma unroll
                    for (int u1 = 0; u1 < U1; u1++) bY[(k1 * 8 + s3_k2) * YR + s3_u0 + 4 * u1] = u[u1];
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 8; k++) v[k] = bY[(s2_k1 * 8 + k) * YR + s2_t0];
            }
            // ---------------- S2 inverse: over k2 -> t1 (into B)
            {
                float2 w[8];
                tw_tmem(twc + 16, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mulc(v[k], w[k]);
            }
            dft8x<true>(v);
#pragma unroll
            for (int n = 0; n < 8; n++) bB[s2_k1 * XR + s2_t0 + T0 * n] = v[n];
            gsync();
            // ---------------- S1 inverse: over k1 -> n, store the row
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = bB[k * XR + t];
            {
                float2 w[8];
                tw_tmem(twc, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mulc(v[k], w[k]);
            }
            dft8x<true>(v);
            float2* dst = reinterpret_cast<float2*>(j.dst);
#pragma unroll
            for (int n = 0; n < 8; n++) stg_stream(dst + t + T * n, v[n]);
        }
        if (sync_after(ri)) team_sync();
        if (fm && leader) {
            if (ri == 0) { __threadfence(); st_release(fb.flags + 2 * strip, fb.epoch); }
            if (ri == 2) st_release(fb.flags + 2 * strip + 1, fb.epoch);
        }
    }
  }
    // a bulk load still in flight (only after an aborted wait) must land before the CTA exits
    if (pending && t == 0) {
        const long long t0c = clock64();
        while (!mbar_try_wait(bar, nld & 1) && clock64() - t0c < kWaitCycles) {}
    }
    tm_fence_before();
    cta_bar();
    tm_fence_after();
    if (!MEGA && warp == 0) tm_dealloc(tbase, G::TMEM_COLS);
}

}  // namespace hyb
