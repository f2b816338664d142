// tm_body.cuh -- the n1 = 4096 fused FP32 advance as a CTA-wide device function, so that the
// kernel of fused_tm.cu and the single-launch batched step (batch_step.cu) run the same code.
//
// Single-pass FP32 hybrid advance for n1 = 4096 with the k1-space lines kept
// in tensor memory (TMEM) and the input rows brought in by
// the bulk-copy engine (TMA).  A CTA sweeps a strip of x2 rows; per row five
// rounds of three real FFTs, one per thread group, with the Faraday and Ampere
// updates of Eqs. hybrid2db1-hybrid2de3 as per-mode epilogues (the schedule of
// tm_sched.cuh, shared with the n1 = 512 .. 2048 kernel of fused_tmt.cu):
//
//   * three groups of T = 256 threads (24 warps per SM); a thread holds 8
//     complex points of a line;
//   * the ten k1-space lines ("slots") live in TMEM: thread t of every group
//     owns the same 8 modes, stored in TMEM lane (t mod 128) at columns
//     (t / 128) * 160 + 16 * slot, so the per-mode updates are lane-local
//     tcgen05.ld / tcgen05.st of 32-bit words;
//   * shared memory holds, per group, the staging row of the next forward
//     transform (one cp.async.bulk of 16 KB, completion on an mbarrier) and
//     two exchange buffers that alternate between consecutive transforms, so
//     a transform needs no barrier after its last exchange; plus the twiddle
//     tables; the per-mode symbols of a thread's modes sit in TMEM beside its
//     slots;
//   * of the three exchanges of a transform only the first and the last cross
//     warps (group barrier); the middle one stays inside a warp.
//
// Real FFT of N = 4096 points: the M = 2048-point complex FFT of
// z[j] = x[2j] + i x[2j+1], factored 8 x 8 x 8 x 4:
//   S1  thread t holds z[t + 256 n], 8-point DFT over n -> k1, twiddle W_2048^{t k1};
//   S2  thread (t0, k1), t = t0 + 32 t1: 8-point DFT over t1 -> k2, twiddle W_256^{t0 k2};
//   S3  thread (u0, k1, k2), t0 = u0 + 4 u1: 8-point DFT over u1 -> k3, twiddle W_32^{u0 k3};
//   S4  thread owns columns c = k1 + 8 k2 + 64 k3 in {t, 512 - t} (t = 0: {0, 256}),
//       4-point DFT over u0 -> Z[c + 512 k4].
// Z[kappa] and Z[M - kappa] then sit in the same thread (columns c and 512 - c),
// so the even/odd split of the real transform is done in registers.  Element
// e = 2 k4 of a thread is mode cA + 512 k4, element e = 2 k4 + 1 is mode
// cB + 512 (3 - k4) = M - (cA + 512 k4); thread 0 stores (X_0, X_M) packed in
// element 0.  The inverse runs the same stages transposed with conjugate
// twiddles.
#pragma once
#include <math.h>

#include "fused_api.cuh"
#include "fused_dev.cuh"
#include "packed_dev.cuh"
#include "tm_dev.cuh"
#include "tm_sched.cuh"

namespace hyb {

namespace tmk {
constexpr int N = 4096, M = 2048, T = 256, NT = 768;
constexpr int XS = 64 * 34;                              // exchange buffer (float2): the S2 -> S3 layout is 64 x 34
constexpr int OFF_STAGE = 0;                             // [3][M] float2
constexpr int OFF_XB = OFF_STAGE + 3 * M * 8;            // [3][2][XS] float2
constexpr int OFF_SYMN = OFF_XB + 3 * 2 * XS * 8;        // float4: the Nyquist mode's symbols
constexpr int OFF_BAR = OFF_SYMN + 16;                   // [3] mbarrier
constexpr int OFF_MISC = OFF_BAR + 3 * 8;                // TMEM base address, abort flag
constexpr int SMEM = OFF_MISC + 16;
constexpr uint32_t TMEM_COLS = 512;                      // slots 2 x 160, symbols 2 x 32, twiddles 2 x 64
constexpr int SYM_COL = 320;                             // per-mode symbols: S (16 words), cj1 (8), cj (8)
// per-thread twiddles (the same for the three groups' thread t): W_2048^{t k} at +0, W_256^{t0 k}
// at +16, W_32^{u0 k} at +32 (k = 1..7, two words each), the split's W_4096^{cA} W_8^{k4} at +48
constexpr int TW_COL = 384;
constexpr long long WAIT_CYCLES = kWaitCycles;            // about 2 s at 2 GHz
}  // namespace tmk

// exchange-buffer position of the S3 -> S4 value of column c = k1 + 8 k2 + 64 k3 and
// u0: inside the 256-entry region k1, which is the region the S2 threads of warp
// k1 read, so S2 -> S3 -> (region reuse) stays inside one warp; the XOR terms keep
// the S3 writes and the S4 reads of column t free of bank conflicts.  The base
// for even u0 is pos(0), for odd u0 pos(1); position(u0) = base + 64 u0.
__device__ __forceinline__ int x3base(int k1, int k2, int k3, int u0odd) {
    return k1 * 256 + 8 * (k3 ^ ((k2 ^ u0odd) & 1)) + (k2 ^ k1);
}
// One CTA of 768 threads (three groups of 256) sweeping the work items vb, vb + vg, ... of fb;
// sm is the CTA's dynamic shared memory (tmk::SMEM bytes).  The whole CTA calls it, and the
// body allocates and frees its 512 TMEM columns itself.
__device__ __forceinline__ void tm_body(const FusedBatch& fb, const int vb, const int vg, unsigned char* sm) {
    using namespace tmk;
    float2* stage = reinterpret_cast<float2*>(sm + OFF_STAGE);
    float2* xbuf = reinterpret_cast<float2*>(sm + OFF_XB);
    float4* symN = reinterpret_cast<float4*>(sm + OFF_SYMN);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(sm + OFF_MISC);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + OFF_MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid / T, t = tid % T;
    const bool fm = fb.flags != nullptr;
    if (vb >= fb.n_items) return;

    // ---- one-time set-up: TMEM, barriers, twiddles
    if (warp == 0) {
        tm_alloc(smem_addr(s_taddr), TMEM_COLS);
        tm_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < 3; k++) mbar_init(smem_addr(bars + k), 1);
        mbar_fence_init();
        *s_abort = 0;
    }
    const FusedInst& i0 = fb.inst[fb.items[vb].x];
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = *s_taddr;
    // this thread's TMEM words: lane t mod 128 (the warp's quarter), columns (t / 128) * 160 + 16 slot + ...
    const uint32_t tw = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((t >> 7) * 160);
    auto ta = [&](int slot, int chunk) { return tw + (uint32_t)(16 * slot + 8 * chunk); };
    // symbols of this thread's modes: S of elements 4c..4c+3 at ts + 8c, cj1 at ts + 16 + 4c, cj at ts + 24 + 4c
    const uint32_t ts = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(SYM_COL + (t >> 7) * 32);

    // modes owned by this thread
    const int cA = t, cB = (t == 0) ? 256 : 512 - t;
    const float2 wA = i0.twC[t];                                     // W_4096^{cA}
    const int qA0 = x3base(cA & 7, (cA >> 3) & 7, cA >> 6, 0), qA1 = x3base(cA & 7, (cA >> 3) & 7, cA >> 6, 1);
    const int qB0 = x3base(cB & 7, (cB >> 3) & 7, cB >> 6, 0), qB1 = x3base(cB & 7, (cB >> 3) & 7, cB >> 6, 1);
    auto kap = [&](int e) { return (e & 1) ? cB + 512 * (3 - (e >> 1)) : cA + 512 * (e >> 1); };
    // stage thread maps
    const int s2_t0 = t & 31, s2_k1 = t >> 5;
    const int s3_k2 = t & 7, s3_u0 = (t >> 3) & 3, s3_k1 = t >> 5;
    const int s3_rd = (s3_k1 * 8 + s3_k2) * 34 + s3_u0;                   // + 4 u1
    // S3 writes of k3: even k3 at s3_we + 16 (k3 / 2), odd k3 at s3_wo + 16 (k3 / 2)
    const int s3_w0 = x3base(s3_k1, s3_k2, 0, s3_u0 & 1) + 64 * s3_u0;
    const int s3_w1 = x3base(s3_k1, s3_k2, 1, s3_u0 & 1) + 64 * s3_u0;
    auto s3_pos = [&](int k3) { return ((k3 & 1) ? s3_w1 : s3_w0) + 16 * (k3 >> 1); };
    auto x3_pos = [&](int q0, int q1, int u0) { return ((u0 & 1) ? q1 : q0) + 64 * u0; };
    constexpr float inv2M = 0.5f / (float)M;

    // this thread's twiddles into TMEM (written by group 0; thread t of every group reads them)
    const uint32_t twc = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(TW_COL + (t >> 7) * 64);
    if (g == 0) {
        float r[16];
        auto put = [&](int step, int i, uint32_t col) {      // W_2048^{step i k}, k = 1..7
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
        put(1, t, 0);
        put(8, s2_t0, 16);
        put(64, s3_u0, 32);
        float q[8];
#pragma unroll
        for (int k4 = 0; k4 < 4; k4++) {
            const float2 w = mul(wA, wr(8, k4));
            q[2 * k4] = w.x;
            q[2 * k4 + 1] = w.y;
        }
        tm_st8(twc + 48, q);
        tm_wait_st();
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();

    const uint32_t bar = smem_addr(bars + g);
    float2* stg = stage + g * M;
    const uint32_t stg_s = smem_addr(stg);
    uint32_t nld = 0;          // bulk loads of this group consumed so far (mbarrier phase)
    int tc = 0;                // transforms of this group so far (exchange-buffer alternation)
    int cur_inst = -1;
    bool pending = false;      // a bulk load issued and not yet consumed

    auto gsync = [&]() { asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(T) : "memory"); };
    auto cta_sync = [&]() { tm_fence_before(); __syncthreads(); tm_fence_after(); };

  for (int item = vb; item < fb.n_items; item += vg) {
    const int4 it = fb.items[item];
    const FusedInst& a = fb.inst[it.x];
    const int strip = it.y, p0 = it.z, p1 = it.w;
    const int H = p1 - p0;
    const int nrounds = 3 + 5 * H;
    const float a2 = a.a2;
    const int next = fm ? (strip + 1) % fb.n_strips : 0;
    const int ri_wait_halo = 3 + 5 * (H - 1);                      // R1 of the last row reads the next strip's copy
    const int ri_wait_read = 3 + 5 * (H - 1) + 3;                  // first write of the last row
    auto cta_sync_after = [&](int ri) {
        if (ri < 3) return ri >= 1 || fm;
        const int r = (ri - 3) % 5;
        return r == 0 || r == 1;
    };
    if (it.x != cur_inst) {
        // per-instance symbols of this thread's modes into TMEM (written once by group 0;
        // the other groups' threads t own the same modes), the Nyquist entry into shared memory
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        if (g == 0) {
            float r[16];
#pragma unroll
            for (int e = 0; e < 8; e++) { const float4 q = a.sym[kap(e)]; r[2 * e] = q.x; r[2 * e + 1] = q.y; }
            tm_st16(ts, r);
#pragma unroll
            for (int e = 0; e < 8; e++) { const float4 q = a.sym[kap(e)]; r[e] = q.z; r[8 + e] = q.w; }
            tm_st16(ts + 16, r);
            tm_wait_st();
        }
        if (tid == 0) *symN = a.sym[M];
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        cur_inst = it.x;
    }
    int fidx = 0;
    // source of this group's next forward transform; the first one is staged now
    bool ndirect = false;
    const float* nsrc = tm_src(a, N, strip, p0, p1, g, 0, fm, next, &ndirect);
    pending = nsrc != nullptr && !ndirect;
    if (pending && t == 0) {
        mbar_expect_tx(bar, 4 * N);
        bulk_load(stg_s, nsrc, 4 * N, bar);
    }

    for (int ri = 0; ri < nrounds; ri++) {
        if (fm && (ri == ri_wait_halo || ri == ri_wait_read)) {
            if (tid == 0) wait_flag(fb.flags + 2 * next + (ri == ri_wait_read ? 1 : 0), fb.epoch, fb.err);
            __syncthreads();
        }
        const Job j = tm_job(a, N, p0, p1, ri, g);
        float2* X = xbuf + (g * 2 + (tc & 1)) * XS;
        float2* Y = xbuf + (g * 2 + ((tc & 1) ^ 1)) * XS;
        if (j.kind == J_FWD) {
            // ---------------- S1: 8-point DFT of z[t + 256 n]
            float2 v[8];
            if (ndirect) {
                const float2* s = reinterpret_cast<const float2*>(nsrc);
#pragma unroll
                for (int n = 0; n < 8; n++) v[n] = ldg_stream(s + t + 256 * n);
            } else {
                mbar_wait(bar, nld & 1, fb.err, s_abort);
                nld++;
                pending = false;
#pragma unroll
                for (int n = 0; n < 8; n++) v[n] = stg[t + 256 * n];
            }
            if (fm && ri == 0 && g != 1) {
                // publish E1 (g = 0) or E3 (g = 2) of the strip's first row for the previous strip
                float2* h = reinterpret_cast<float2*>(const_cast<float*>(a.halo) + ((size_t)strip * 7 + (g == 0 ? 0 : 1)) * N);
#pragma unroll
                for (int n = 0; n < 8; n++) h[t + 256 * n] = v[n];
            }
            dft8x<false>(v);
            {
                float2 w[8];
                tw_tmem(twc, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mul(v[k], w[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; k++) X[k * 256 + t] = v[k];
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
            // ---------------- S2
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = X[s2_k1 * 256 + s2_t0 + 32 * n];
            dft8x<false>(v);
            {
                float2 w[8];
                tw_tmem(twc + 16, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mul(v[k], w[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; k++) Y[(s2_k1 * 8 + k) * 34 + s2_t0] = v[k];
            __syncwarp();                     // S2 -> S3 stays inside the warp (k1 = warp)
            // ---------------- S3
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = Y[s3_rd + 4 * n];
            dft8x<false>(v);
            {
                float2 w[8];
                tw_tmem(twc + 32, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mul(v[k], w[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; k++) X[s3_pos(k)] = v[k];
            gsync();
            // ---------------- S4: columns cA, cB, 4-point DFT over u0
            float2 A[4], Bc[4];
#pragma unroll
            for (int u = 0; u < 4; u++) { A[u] = X[x3_pos(qA0, qA1, u)]; Bc[u] = X[x3_pos(qB0, qB1, u)]; }
            dft4x<false>(A[0], A[1], A[2], A[3]);
            dft4x<false>(Bc[0], Bc[1], Bc[2], Bc[3]);
            tc++;
            // even/odd split into the real-input coefficients of this thread's modes
            float2 x[8];
            {
                float ws[8];
                tm_ld8(twc + 48, ws);
                tm_wait_ld();
#pragma unroll
                for (int k4 = 0; k4 < 4; k4++) split_fwd(A[k4], Bc[3 - k4], f2(ws[2 * k4], ws[2 * k4 + 1]), x[2 * k4], x[2 * k4 + 1]);
            }
            if (t == 0) {
                // columns 0 and 256 pair with themselves: Z[0] gives (X_0, X_M), Z[512] with
                // Z[1536], Z[1024] with itself, Z[256] with Z[1792], Z[768] with Z[1280]
                x[0] = f2(A[0].x + A[0].y, A[0].x - A[0].y);
                split_fwd(A[1], A[3], wconst<8, 1, false>(), x[2], x[6]);
                float2 dummy;
                split_fwd(A[2], A[2], wconst<4, 1, false>(), x[4], dummy);
                split_fwd(Bc[0], Bc[3], wconst<16, 1, false>(), x[7], x[1]);
                split_fwd(Bc[1], Bc[2], wconst<16, 3, false>(), x[5], x[3]);
            }
            // ---------------- epilogue: per-mode updates, two chunks of four modes
            tm_epilogue(j, x, tw, ts, symN, a2, t == 0);
        } else if (j.kind == J_INV) {
            // ---------------- slot -> inverse split -> inverse 4-point DFT over k4
            float2 x[8];
#pragma unroll
            for (int c = 0; c < 2; c++) {
                float r[8];
                tm_ld8(ta(j.slot, c), r);
                tm_wait_ld();
#pragma unroll
                for (int i = 0; i < 4; i++) x[4 * c + i] = f2(r[2 * i], r[2 * i + 1]);
            }
            float2 A[4], Bc[4];
            {
                float ws[8];
                tm_ld8(twc + 48, ws);
                tm_wait_ld();
#pragma unroll
                for (int k4 = 0; k4 < 4; k4++) split_inv(x[2 * k4], x[2 * k4 + 1], f2(ws[2 * k4], ws[2 * k4 + 1]), inv2M, A[k4], Bc[3 - k4]);
            }
            if (t == 0) {
                A[0] = f2((x[0].x + x[0].y) * inv2M, (x[0].x - x[0].y) * inv2M);
                split_inv(x[2], x[6], wconst<8, 1, false>(), inv2M, A[1], A[3]);
                float2 dummy;
                split_inv(x[4], x[4], wconst<4, 1, false>(), inv2M, A[2], dummy);
                split_inv(x[7], x[1], wconst<16, 1, false>(), inv2M, Bc[0], Bc[3]);
                split_inv(x[5], x[3], wconst<16, 3, false>(), inv2M, Bc[1], Bc[2]);
            }
            dft4x<true>(A[0], A[1], A[2], A[3]);
            dft4x<true>(Bc[0], Bc[1], Bc[2], Bc[3]);
#pragma unroll
            for (int u = 0; u < 4; u++) { X[x3_pos(qA0, qA1, u)] = A[u]; X[x3_pos(qB0, qB1, u)] = Bc[u]; }
            gsync();
            // ---------------- S3 inverse: twiddle, inverse 8-point DFT over k3 -> u1
            float2 v[8];
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = X[s3_pos(k)];
            {
                float2 w[8];
                tw_tmem(twc + 32, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mulc(v[k], w[k]);
            }
            dft8x<true>(v);
#pragma unroll
            for (int n = 0; n < 8; n++) Y[s3_rd + 4 * n] = v[n];
            __syncwarp();                     // S3 -> S2 inverse stays inside the warp
            // ---------------- S2 inverse: over k2 -> t1
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = Y[(s2_k1 * 8 + k) * 34 + s2_t0];
            {
                float2 w[8];
                tw_tmem(twc + 16, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mulc(v[k], w[k]);
            }
            dft8x<true>(v);
#pragma unroll
            for (int n = 0; n < 8; n++) X[s2_k1 * 256 + s2_t0 + 32 * n] = v[n];
            gsync();
            // ---------------- S1 inverse: over k1 -> n, store the row
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = X[k * 256 + t];
            {
                float2 w[8];
                tw_tmem(twc, w);
#pragma unroll
                for (int k = 1; k < 8; k++) v[k] = mulc(v[k], w[k]);
            }
            dft8x<true>(v);
            float2* dst = reinterpret_cast<float2*>(j.dst);
#pragma unroll
            for (int n = 0; n < 8; n++) stg_stream(dst + t + 256 * n, v[n]);
            tc++;
        }
        if (cta_sync_after(ri)) cta_sync();
        if (fm && tid == 0) {
            if (ri == 0) { __threadfence(); st_release(fb.flags + 2 * strip, fb.epoch); }
            if (ri == 2) st_release(fb.flags + 2 * strip + 1, fb.epoch);
        }
    }
  }
    // a bulk load still in flight (only after an aborted wait) must land before the CTA exits
    if (pending && t == 0) {
        const long long t0 = clock64();
        while (!mbar_try_wait(bar, nld & 1) && clock64() - t0 < WAIT_CYCLES) {}
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(tbase, TMEM_COLS);
}

}  // namespace hyb
