// fused_tm.cu -- single-pass FP32 hybrid advance for n1 = 4096 with the
// k1-space lines kept in tensor memory (TMEM) and the input rows brought in by
// the bulk-copy engine (TMA).  Same schedule as the shared-memory kernel of
// fused2d.cu (a CTA sweeps a strip of x2 rows; per row five rounds of three
// real FFTs, one per thread group, with the Faraday and Ampere updates of
// Eqs. hybrid2db1-hybrid2de3 as per-mode epilogues), re-laid for more warps:
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
//     and per-mode symbol tables.
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
#include <math.h>

#include <vector>

#include "fused_dev.cuh"

namespace hyb {

namespace tmk {
constexpr int N = 4096, M = 2048, T = 256, NT = 768;
constexpr int XS = 64 * 34;                              // exchange buffer (float2): the S2 -> S3 layout is 64 x 34
constexpr int OFF_STAGE = 0;                             // [3][M] float2
constexpr int OFF_XB = OFF_STAGE + 3 * M * 8;            // [3][2][XS] float2
constexpr int OFF_TW1 = OFF_XB + 3 * 2 * XS * 8;         // [7][256] float2  W_2048^{t k1}, k1 = 1..7
constexpr int OFF_TW2 = OFF_TW1 + 7 * 256 * 8;           // [8][32] float2   W_256^{t0 k2}
constexpr int OFF_TW3 = OFF_TW2 + 8 * 32 * 8;            // [8][4] float2    W_32^{u0 k3}
constexpr int OFF_SYM = OFF_TW3 + 8 * 4 * 8;             // [M + 1] float4
constexpr int OFF_BAR = (OFF_SYM + (M + 1) * 16 + 7) / 8 * 8;   // [3] mbarrier
constexpr int OFF_MISC = OFF_BAR + 3 * 8;                // TMEM base address, abort flag
constexpr int SMEM = OFF_MISC + 16;
constexpr uint32_t TMEM_COLS = 512;                      // 2 x 160 used
constexpr long long WAIT_CYCLES = 4000000000LL;          // about 2 s at 2 GHz
}  // namespace tmk

// ------------------------------------------------------------------ TMEM, mbarrier and bulk-copy primitives
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tm_alloc(uint32_t dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
// 32 lanes x 8 columns of 32 bits: this thread's lane, 8 consecutive words
__device__ __forceinline__ void tm_ld8(uint32_t ta, float (&r)[8]) {
    uint32_t u[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                 : "r"(ta));
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tm_st8(uint32_t ta, const float (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "r"(ta), "r"(__float_as_uint(r[0])), "r"(__float_as_uint(r[1])), "r"(__float_as_uint(r[2])),
                    "r"(__float_as_uint(r[3])), "r"(__float_as_uint(r[4])), "r"(__float_as_uint(r[5])),
                    "r"(__float_as_uint(r[6])), "r"(__float_as_uint(r[7]))
                 : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) global -> shared
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait for phase `parity` of an mbarrier; on time-out sets bit 1 of *err
// and the CTA's abort flag (later waits then return at once)
__device__ __forceinline__ void mbar_wait(uint32_t bar, uint32_t parity, int* err, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return;
        if (clock64() - t0 > tmk::WAIT_CYCLES) {
            if (err) atomicOr(err, 2);
            *abort_flag = 1;
            return;
        }
    }
}

// exchange-buffer position of the S3 -> S4 value (column c, u0): XOR swizzle of
// the low four bits keeps both access patterns free of bank conflicts
__device__ __forceinline__ int x3sw(int c) { return c ^ ((c >> 3) & 7); }
__device__ __forceinline__ int x3pos(int csw, int u0) { return u0 * 512 + (csw ^ ((u0 & 1) << 3)); }

// forward split of one pair: X[k] = e - u, X[M-k] = conj(e + u), e = (a + conj b)/2,
// u = (i/2) w (a - conj b), w = W_N^k, a = Z[k], b = Z[M-k]
__device__ __forceinline__ void split_fwd(float2 av, float2 bv, float2 w, float2& xk, float2& xmk) {
    const float2 e = scl(add(av, conjf2(bv)), 0.5f);
    const float2 wd = mul(w, sub(av, conjf2(bv)));
    const float2 u = f2(-0.5f * wd.y, 0.5f * wd.x);
    xk = sub(e, u);
    xmk = conjf2(add(e, u));
}
// inverse split of one pair (with the 1/M of the inverse transform folded in):
// Z[k] = E + iO, Z[M-k] = conj(E - iO), E = (X[k] + conj X[M-k])/2M,
// O = conj(w) (X[k] - conj X[M-k])/2M
__device__ __forceinline__ void split_inv(float2 xa, float2 xbv, float2 w, float s, float2& zk, float2& zmk) {
    const float2 E = scl(add(xa, conjf2(xbv)), s);
    const float2 O = scl(mulc(sub(xa, conjf2(xbv)), w), s);
    const float2 v = f2(-O.y, O.x);
    zk = add(E, v);
    zmk = conjf2(sub(E, v));
}

__global__ void __launch_bounds__(tmk::NT, 1) k_fused_tm(FusedBatch fb) {
    using namespace tmk;
    extern __shared__ __align__(128) unsigned char sm[];
    float2* stage = reinterpret_cast<float2*>(sm + OFF_STAGE);
    float2* xbuf = reinterpret_cast<float2*>(sm + OFF_XB);
    float2* tw1 = reinterpret_cast<float2*>(sm + OFF_TW1);
    float2* tw2 = reinterpret_cast<float2*>(sm + OFF_TW2);
    float2* tw3 = reinterpret_cast<float2*>(sm + OFF_TW3);
    float4* sym = reinterpret_cast<float4*>(sm + OFF_SYM);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(sm + OFF_MISC);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + OFF_MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid / T, t = tid % T;
    const bool fm = fb.flags != nullptr;
    if ((int)blockIdx.x >= fb.n_items) return;

    // ---- one-time set-up: TMEM, barriers, twiddle tables
    if (warp == 0) {
        tm_alloc(smem_addr(s_taddr), TMEM_COLS);
        tm_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < 3; k++) mbar_init(smem_addr(bars + k), 1);
        mbar_fence_init();
        *s_abort = 0;
    }
    const FusedInst& i0 = fb.inst[fb.items[blockIdx.x].x];
    for (int i = tid; i < 7 * 256; i += NT) tw1[i] = i0.twM[(i & 255) * ((i >> 8) + 1)];
    for (int i = tid; i < 8 * 32; i += NT) tw2[i] = i0.twM[8 * (i & 31) * (i >> 5)];
    for (int i = tid; i < 8 * 4; i += NT) tw3[i] = i0.twM[64 * (i & 3) * (i >> 2)];
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = *s_taddr;
    // this thread's TMEM words: lane t mod 128 (the warp's quarter), columns (t / 128) * 160 + 16 slot + ...
    const uint32_t tw = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((t >> 7) * 160);
    auto ta = [&](int slot, int chunk) { return tw + (uint32_t)(16 * slot + 8 * chunk); };

    // modes owned by this thread
    const int cA = t, cB = (t == 0) ? 256 : 512 - t;
    const float2 wA = i0.twC[t];                                     // W_4096^{cA}
    const int cAs = x3sw(cA), cBs = x3sw(cB);
    auto kap = [&](int e) { return (e & 1) ? cB + 512 * (3 - (e >> 1)) : cA + 512 * (e >> 1); };
    // stage thread maps
    const int s2_t0 = t & 31, s2_k1 = t >> 5;
    const int s3_k2 = t & 7, s3_u0 = (t >> 3) & 3, s3_k1 = t >> 5;
    const int s3_rd = (s3_k1 * 8 + s3_k2) * 34 + s3_u0;                   // + 4 u1
    const int s3_wr = x3pos(x3sw(s3_k1 + 8 * s3_k2), s3_u0);             // + 64 k3
    constexpr float inv2M = 0.5f / (float)M;

    const uint32_t bar = smem_addr(bars + g);
    float2* stg = stage + g * M;
    const uint32_t stg_s = smem_addr(stg);
    uint32_t nld = 0;          // bulk loads of this group consumed so far (mbarrier phase)
    int tc = 0;                // transforms of this group so far (exchange-buffer alternation)
    int cur_inst = -1;
    bool pending = false;      // a bulk load issued and not yet consumed

    auto gsync = [&]() { asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(T) : "memory"); };
    auto cta_sync = [&]() { tm_fence_before(); __syncthreads(); tm_fence_after(); };

  for (int item = blockIdx.x; item < fb.n_items; item += gridDim.x) {
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
        return r == 0 || r == 1 || r == 4;
    };
    // the forward source read directly (not staged): the next strip's published copy
    auto is_direct = [&](int idx) {
        if (!fm) return false;
        const int npro = (g == 0) ? 3 : 2;
        if (idx < npro || g == 2) return false;
        const int q = idx - npro;
        return (q % 3) == 0 && p0 + q / 3 + 1 == p1;
    };
    if (it.x != cur_inst) {                                       // per-instance symbol table
        __syncthreads();
        for (int i = tid; i <= M; i += NT) sym[i] = a.sym[i];
        __syncthreads();
        cur_inst = it.x;
    }
    int fidx = 0;
    // first staged row of this item
    if (t == 0) {
        const float* s0 = fwd_src(a, N, strip, p0, p1, g, 0, fm, next);
        if (s0 && !is_direct(0)) {
            mbar_expect_tx(bar, 4 * N);
            bulk_load(stg_s, s0, 4 * N, bar);
        }
    }
    pending = !is_direct(0) && fwd_src(a, N, strip, p0, p1, g, 0, fm, next) != nullptr;

    for (int ri = 0; ri < nrounds; ri++) {
        if (fm && (ri == ri_wait_halo || ri == ri_wait_read)) {
            if (tid == 0) wait_flag(fb.flags + 2 * next + (ri == ri_wait_read ? 1 : 0), fb.epoch, fb.err);
            __syncthreads();
        }
        const Job j = job_of(a, N, strip, p0, p1, ri, g);
        float2* X = xbuf + (g * 2 + (tc & 1)) * XS;
        float2* Y = xbuf + (g * 2 + ((tc & 1) ^ 1)) * XS;
        if (j.kind == J_FWD) {
            // ---------------- S1: 8-point DFT of z[t + 256 n]
            float2 v[8];
            if (is_direct(fidx)) {
                const float2* s = reinterpret_cast<const float2*>(fwd_src(a, N, strip, p0, p1, g, fidx, fm, next));
#pragma unroll
                for (int n = 0; n < 8; n++) v[n] = ldg_stream(s + t + 256 * n);
            } else {
                mbar_wait(bar, nld & 1, fb.err, s_abort);
                nld++;
                pending = false;
#pragma unroll
                for (int n = 0; n < 8; n++) v[n] = stg[t + 256 * n];
            }
            if (fm && ri == 0 && g < 2) {
                // publish E1 (g = 0) or E3 (g = 1) of the strip's first row for the previous strip
                float2* h = reinterpret_cast<float2*>(const_cast<float*>(a.halo) + ((size_t)strip * 7 + g) * N);
#pragma unroll
                for (int n = 0; n < 8; n++) h[t + 256 * n] = v[n];
            }
            Dft<8, false>::run(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = mul(v[k], tw1[(k - 1) * 256 + t]);
#pragma unroll
            for (int k = 0; k < 8; k++) X[k * 256 + t] = v[k];
            gsync();
            fidx++;
            // the group's staging row is free: start the next forward's row
            {
                const float* ns = fwd_src(a, N, strip, p0, p1, g, fidx, fm, next);
                const bool go = ns != nullptr && !is_direct(fidx);
                if (go && t == 0) {
                    fence_proxy_async_smem();
                    mbar_expect_tx(bar, 4 * N);
                    bulk_load(stg_s, ns, 4 * N, bar);
                }
                pending = go;
            }
            // ---------------- S2
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = X[s2_k1 * 256 + s2_t0 + 32 * n];
            Dft<8, false>::run(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = mul(v[k], tw2[k * 32 + s2_t0]);
#pragma unroll
            for (int k = 0; k < 8; k++) Y[(s2_k1 * 8 + k) * 34 + s2_t0] = v[k];
            gsync();
            // ---------------- S3
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = Y[s3_rd + 4 * n];
            Dft<8, false>::run(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = mul(v[k], tw3[k * 4 + s3_u0]);
#pragma unroll
            for (int k = 0; k < 8; k++) X[s3_wr + 64 * k] = v[k];
            gsync();
            // ---------------- S4: columns cA, cB, 4-point DFT over u0
            float2 A[4], Bc[4];
#pragma unroll
            for (int u = 0; u < 4; u++) { A[u] = X[x3pos(cAs, u)]; Bc[u] = X[x3pos(cBs, u)]; }
            Dft<4, false>::run(A);
            Dft<4, false>::run(Bc);
            tc++;
            // even/odd split into the real-input coefficients of this thread's modes
            float2 x[8];
#pragma unroll
            for (int k4 = 0; k4 < 4; k4++) split_fwd(A[k4], Bc[3 - k4], mul(wA, wr(8, k4)), x[2 * k4], x[2 * k4 + 1]);
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
            const int p = j.row;
            const int ds = j.slot;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                float o[8];
                const int e0 = 4 * c;
                switch (j.epi) {
                case X_STORE:
#pragma unroll
                    for (int i = 0; i < 4; i++) { o[2 * i] = x[e0 + i].x; o[2 * i + 1] = x[e0 + i].y; }
                    break;
                case X_B1: {        // B1 -= a2 (E3(p+1) - E3(p))
                    float u[8], w[8];
                    tm_ld8(ta(sE3(p + 1), c), u);
                    tm_ld8(ta(sE3(p), c), w);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        o[2 * i] = x[e0 + i].x - a2 * (u[2 * i] - w[2 * i]);
                        o[2 * i + 1] = x[e0 + i].y - a2 * (u[2 * i + 1] - w[2 * i + 1]);
                    }
                } break;
                case X_B2: {        // B2 += S E3(p)
                    float w[8];
                    tm_ld8(ta(sE3(p), c), w);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float4 q = sym[kap(e0 + i)];
                        const float2 r = add(x[e0 + i], mul(f2(q.x, q.y), f2(w[2 * i], w[2 * i + 1])));
                        o[2 * i] = r.x; o[2 * i + 1] = r.y;
                    }
                    if (c == 0 && t == 0) {   // packed DC/Nyquist: two real updates
                        o[0] = x[0].x + sym[0].x * w[0];
                        o[1] = x[0].y + sym[M].x * w[1];
                    }
                } break;
                case X_B3: {        // B3 += a2 (E1(p+1) - E1(p)) - S E2(p)
                    float u[8], w[8], e2[8];
                    tm_ld8(ta(sE1(p + 1), c), u);
                    tm_ld8(ta(sE1(p), c), w);
                    tm_ld8(ta(sE2, c), e2);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float4 q = sym[kap(e0 + i)];
                        const float2 se = mul(f2(q.x, q.y), f2(e2[2 * i], e2[2 * i + 1]));
                        o[2 * i] = x[e0 + i].x + a2 * (u[2 * i] - w[2 * i]) - se.x;
                        o[2 * i + 1] = x[e0 + i].y + a2 * (u[2 * i + 1] - w[2 * i + 1]) - se.y;
                    }
                    if (c == 0 && t == 0) {
                        o[0] = x[0].x + a2 * (u[0] - w[0]) - sym[0].x * e2[0];
                        o[1] = x[0].y + a2 * (u[1] - w[1]) - sym[M].x * e2[1];
                    }
                } break;
                case X_J1: {        // E1 += a2 (B3(p) - B3(p-1)) - cj1 j1
                    float u[8], w[8], d[8];
                    tm_ld8(ta(sB3(p), c), u);
                    tm_ld8(ta(sB3(p - 1), c), w);
                    tm_ld8(ta(ds, c), d);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float cj1 = sym[kap(e0 + i)].z;
                        o[2 * i] = d[2 * i] + a2 * (u[2 * i] - w[2 * i]) - cj1 * x[e0 + i].x;
                        o[2 * i + 1] = d[2 * i + 1] + a2 * (u[2 * i + 1] - w[2 * i + 1]) - cj1 * x[e0 + i].y;
                    }
                    if (c == 0 && t == 0) o[1] = d[1] + a2 * (u[1] - w[1]) - sym[M].z * x[0].y;
                } break;
                case X_J2: {        // E2 += conj(S) B3(p) - cj j2
                    float u[8], d[8];
                    tm_ld8(ta(sB3(p), c), u);
                    tm_ld8(ta(ds, c), d);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float4 q = sym[kap(e0 + i)];
                        const float2 sb = mulc(f2(u[2 * i], u[2 * i + 1]), f2(q.x, q.y));
                        o[2 * i] = d[2 * i] + sb.x - q.w * x[e0 + i].x;
                        o[2 * i + 1] = d[2 * i + 1] + sb.y - q.w * x[e0 + i].y;
                    }
                    if (c == 0 && t == 0) {
                        const float4 qd = sym[0], qn = sym[M];
                        o[0] = d[0] + qd.x * u[0] - qd.w * x[0].x;
                        o[1] = d[1] + qn.x * u[1] - qn.w * x[0].y;
                    }
                } break;
                default: {          // X_J3: E3 += -conj(S) B2(p) - a2 (B1(p) - B1(p-1)) - cj j3
                    float b2[8], u[8], w[8], d[8];
                    tm_ld8(ta(sB2, c), b2);
                    tm_ld8(ta(sB1(p), c), u);
                    tm_ld8(ta(sB1(p - 1), c), w);
                    tm_ld8(ta(ds, c), d);
                    tm_wait_ld();
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float4 q = sym[kap(e0 + i)];
                        const float2 sb = mulc(f2(b2[2 * i], b2[2 * i + 1]), f2(q.x, q.y));
                        o[2 * i] = d[2 * i] - sb.x - a2 * (u[2 * i] - w[2 * i]) - q.w * x[e0 + i].x;
                        o[2 * i + 1] = d[2 * i + 1] - sb.y - a2 * (u[2 * i + 1] - w[2 * i + 1]) - q.w * x[e0 + i].y;
                    }
                    if (c == 0 && t == 0) {
                        const float4 qd = sym[0], qn = sym[M];
                        o[0] = d[0] - qd.x * b2[0] - a2 * (u[0] - w[0]) - qd.w * x[0].x;
                        o[1] = d[1] - qn.x * b2[1] - a2 * (u[1] - w[1]) - qn.w * x[0].y;
                    }
                } break;
                }
                tm_st8(ta(ds, c), o);
            }
            tm_wait_st();
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
#pragma unroll
            for (int k4 = 0; k4 < 4; k4++) split_inv(x[2 * k4], x[2 * k4 + 1], mul(wA, wr(8, k4)), inv2M, A[k4], Bc[3 - k4]);
            if (t == 0) {
                A[0] = f2((x[0].x + x[0].y) * inv2M, (x[0].x - x[0].y) * inv2M);
                split_inv(x[2], x[6], wconst<8, 1, false>(), inv2M, A[1], A[3]);
                float2 dummy;
                split_inv(x[4], x[4], wconst<4, 1, false>(), inv2M, A[2], dummy);
                split_inv(x[7], x[1], wconst<16, 1, false>(), inv2M, Bc[0], Bc[3]);
                split_inv(x[5], x[3], wconst<16, 3, false>(), inv2M, Bc[1], Bc[2]);
            }
            Dft<4, true>::run(A);
            Dft<4, true>::run(Bc);
#pragma unroll
            for (int u = 0; u < 4; u++) { X[x3pos(cAs, u)] = A[u]; X[x3pos(cBs, u)] = Bc[u]; }
            gsync();
            // ---------------- S3 inverse: twiddle, inverse 8-point DFT over k3 -> u1
            float2 v[8];
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = X[s3_wr + 64 * k];
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = mulc(v[k], tw3[k * 4 + s3_u0]);
            Dft<8, true>::run(v);
#pragma unroll
            for (int n = 0; n < 8; n++) Y[s3_rd + 4 * n] = v[n];
            gsync();
            // ---------------- S2 inverse: over k2 -> t1
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = Y[(s2_k1 * 8 + k) * 34 + s2_t0];
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = mulc(v[k], tw2[k * 32 + s2_t0]);
            Dft<8, true>::run(v);
#pragma unroll
            for (int n = 0; n < 8; n++) X[s2_k1 * 256 + s2_t0 + 32 * n] = v[n];
            gsync();
            // ---------------- S1 inverse: over k1 -> n, store the row
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = X[k * 256 + t];
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = mulc(v[k], tw1[(k - 1) * 256 + t]);
            Dft<8, true>::run(v);
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

// ------------------------------------------------------------------ host side
size_t fused_tm_smem_bytes() { return (size_t)tmk::SMEM; }

cudaError_t fused_tm_occupancy(int* occ) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_tm, cudaFuncAttributeMaxDynamicSharedMemorySize, tmk::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_fused_tm, tmk::NT, tmk::SMEM);
    if (e == cudaSuccess && *occ > 1) *occ = 1;     // TMEM holds one CTA's lines per SM
    return e;
}

cudaError_t fused_tm_launch(const FusedBatch& fb, int grid, cudaStream_t s) {
    if (fb.flags) {
        void* args[] = {const_cast<FusedBatch*>(&fb)};
        return cudaLaunchCooperativeKernel((const void*)k_fused_tm, dim3(grid), dim3(tmk::NT), args, tmk::SMEM, s);
    }
    k_fused_tm<<<grid, tmk::NT, tmk::SMEM, s>>>(fb);
    return cudaGetLastError();
}

}  // namespace hyb
