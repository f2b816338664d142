// fused2d.cu -- single-pass FP32 hybrid advance for 2D grids with
// n1 in {512, 1024, 2048} (n1 = 4096 runs the TMEM kernel of fused_tm.cu, which
// shares the host side below): one kernel reads E^n, B^{n-1/2}, j^{n+1/2}
// once from HBM and writes E^{n+1}, B^{n+1/2} once (15 words per cell).
//
// Work decomposition.  The Faraday/Ampere updates of Eqs. hybrid2db1-de3 are
// pointwise in the x1 mode kappa and couple only neighbouring x2 rows, so each
// CTA sweeps a strip of consecutive x2 rows, keeping the k1-space lines it
// still needs in shared memory ("slots"): E1, E3 of rows p and p+1, E2 of row
// p, B1, B3 of rows p-1 and p, B2 of row p (10 lines).  Rows just outside the
// strip (E, B1, B3 of row p0-1; E1, E3 of row p1) are either exchanged inside
// the kernel under release/acquire flags (one co-resident CTA per strip) or
// copied each step by a small kernel into a halo buffer before any CTA
// overwrites them (batches).
//
// The CTA has three thread groups of T = n1/32 threads; in every "round" each
// group performs one real FFT of one row (forward or inverse), so the three
// groups run in lock-step and share __syncthreads:
//   R1  FFT E1(p+1), E3(p+1), E2(p)                            -> slots
//   R2  FFT B1(p), B2(p), B3(p); Faraday update                 -> slots
//   R3  FFT j1(p), j2(p), j3(p); j1 correction, filter, Ampere  -> E slots
//   R4  inverse FFT E1(p), E2(p), E3(p)                         -> HBM
//   R5  inverse FFT B1(p), B2(p), B3(p)                         -> HBM
//
// Real FFT of n1 = N points: the N/2 = M-point complex FFT of
// z[j] = x[2j] + i x[2j+1], factored M = 16 * 16 * P3 (P3 = T/16):
//   stage 1: thread n_a = t holds z[t + T n_b], 16-point DFT over n_b, twiddle W_M^{t k_b};
//   stage 2: thread (k_b, m_a) gathers 16 values over m_b from shared memory,
//            16-point DFT, twiddle W_T^{m_a l_b};
//   stage 3: thread gathers P3 values of a column c = k_b + 16 l_b, P3-point DFT
//            -> Z[c + 256 l_a].
// Each thread owns column pairs {c, 256 - c}, so the even/odd split that turns
// Z into the N/2+1 real-input coefficients X (it pairs kappa with M - kappa)
// happens in registers; a thread owns the same set of kappa for every line,
// so the per-mode updates are thread-local reads and writes of slots.  The
// DC and Nyquist coefficients (both real) are packed into one complex slot.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fused_dev.cuh"

namespace hyb {



template <int N>
struct Geo {
    static constexpr int M = N / 2;
    static constexpr int T = M / 16;
    static constexpr int P3 = T / 16;
    static constexpr int Q = 16 / P3;       // columns per thread
    static constexpr int NT = 3 * T;
    static constexpr int XB = M + 16;       // exchange buffer (float2) per group
    static constexpr int MINB = (N == 4096) ? 1 : (N == 2048) ? 2 : (N == 1024) ? 4 : 6;   // CTAs per SM to fit
};

template <int N>
__global__ void __launch_bounds__(Geo<N>::NT, Geo<N>::MINB) k_fused2d(FusedBatch fb) {
    using G = Geo<N>;
    constexpr int M = G::M, T = G::T, P3 = G::P3, Q = G::Q, XB = G::XB;
    extern __shared__ __align__(16) float2 smem[];
    float2* slots = smem;
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    float2* xb = smem + kSlots * M + g * XB;
    float2* s_tw2 = smem + kSlots * M + 3 * XB;                     // [P3][16] W_T^{ma l}
    if ((int)blockIdx.x >= fb.n_items) return;
    const bool fm = fb.flags != nullptr;

    // twiddles: exact FP64-rounded values, identical for every instance with this n1
    const FusedInst& i0 = fb.inst[fb.items[blockIdx.x].x];
    float2 tw1[16];
    const int kb = t & 15, ma = t >> 4;
#pragma unroll
    for (int k = 0; k < 16; k++) tw1[k] = i0.twM[t * k];         // W_M^{t k}, t k < M
    for (int i = threadIdx.x; i < P3 * 16; i += blockDim.x) s_tw2[i] = i0.twM[16 * (i >> 4) * (i & 15)];
    // column pairs owned by this thread
    int cA[Q / 2];
    float2 wA[Q / 2];
#pragma unroll
    for (int p = 0; p < Q / 2; p++) {
        const int pi = t + T * p;
        cA[p] = pi;
        wA[p] = i0.twC[pi];                                          // W_N^{cA}
    }
    const float2 w128 = i0.twC[128];
    auto colB = [&](int p) { return cA[p] == 0 ? 128 : 256 - cA[p]; };
    const float inv2M = 0.5f / (float)M;
    // Barriers: the three exchanges of a row FFT stay inside a group (named barrier
    // 1 + g over its T threads); the whole CTA synchronises only where slots pass
    // between groups: after P2, P3 (and P1 in flag mode), and after R1, R2, R5.
    auto gsync = [&]() {
        if (T >= 32) asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(T) : "memory");
        else __syncthreads();
    };
    // slot layout: element pairs (e, e+1) of a thread are adjacent (one 16-byte access)
    auto sidx = [&](int sl, int e) { return sl * M + (e >> 1) * (2 * T) + 2 * t + (e & 1); };
    auto ld1 = [&](int sl, int e) { return slots[sidx(sl, e)]; };
    auto ld2 = [&](int sl, int e) { return *reinterpret_cast<const float4*>(slots + sidx(sl, e)); };
    auto st2 = [&](int sl, int e, float2 u, float2 v) {
        *reinterpret_cast<float4*>(slots + sidx(sl, e)) = make_float4(u.x, u.y, v.x, v.y);
    };
    __syncthreads();

  for (int item = blockIdx.x; item < fb.n_items; item += gridDim.x) {
    const int4 it = fb.items[item];
    const FusedInst& a = fb.inst[it.x];
    const int strip = it.y, p0 = it.z, p1 = it.w;
    const int H = p1 - p0;
    const int nrounds = 3 + 5 * H;
    const float a2 = a.a2;
    const int next = fm ? (strip + 1) % fb.n_strips : 0;
    const int ri_wait_halo = 3 + 5 * (H - 2) + 2;                  // round that prefetches the next strip's copy
    const int ri_wait_read = 3 + 5 * (H - 1) + 3;                  // first write of the last row
    auto cta_sync_after = [&](int ri) {
        if (ri < 3) return ri >= 1 || fm;
        const int r = (ri - 3) % 5;
        return r == 0 || r == 1 || r == 4;
    };

    float2 pf[16];
    int fidx = 0;
    {
        const float2* s0 = reinterpret_cast<const float2*>(fwd_src(a, N, strip, p0, p1, g, 0, fm, next));
#pragma unroll
        for (int nb = 0; nb < 16; nb++) pf[nb] = ldg_stream(s0 + t + T * nb);
    }

    float2 x[16];
    for (int ri = 0; ri < nrounds; ri++) {
        if (fm && (ri == ri_wait_halo || ri == ri_wait_read)) {
            if (threadIdx.x == 0) wait_flag(fb.flags + 2 * next + (ri == ri_wait_read ? 1 : 0), fb.epoch, fb.err);
            __syncthreads();
        }
        const Job j = job_of(a, N, strip, p0, p1, ri, g);
        if (j.kind == J_FWD) {
            // ---------------- stage 1: 16-point DFT of z[t + T n_b] from the prefetched row
#pragma unroll
            for (int nb = 0; nb < 16; nb++) x[nb] = pf[nb];
            if (fm && ri == 0 && g < 2) {
                // publish E1 (g = 0) or E3 (g = 1) of the strip's first row for the previous strip
                float2* h = reinterpret_cast<float2*>(const_cast<float*>(a.halo) + ((size_t)strip * 7 + g) * N);
#pragma unroll
                for (int nb = 0; nb < 16; nb++) h[t + T * nb] = x[nb];
            }
            {
                const float2* nsrc = reinterpret_cast<const float2*>(fwd_src(a, N, strip, p0, p1, g, ++fidx, fm, next));
                if (nsrc) {
#pragma unroll
                    for (int nb = 0; nb < 16; nb++) pf[nb] = ldg_stream(nsrc + t + T * nb);
                }
            }
            Dft<16, false>::run(x);
#pragma unroll
            for (int k = 1; k < 16; k++) x[k] = mul(x[k], tw1[k]);
#pragma unroll
            for (int k = 0; k < 16; k++) xb[k * (T + 1) + t] = x[k];
        } else if (j.kind == J_INV) {
            // ---------------- inverse: slot -> pre-processing -> stage 3 inverse
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float4 v = ld2(j.slot, e);
                x[e] = f2(v.x, v.y);
                x[e + 1] = f2(v.z, v.w);
            }
            // pair pre-processing: Z[k] = E + iO, Z[M-k] = conj(E - iO)
#pragma unroll
            for (int p = 0; p < Q / 2; p++) {
#pragma unroll
                for (int l = 0; l < P3; l++) {
                    const int ea = (2 * p) * P3 + l;
                    const int eb = (2 * p + 1) * P3 + (P3 - 1 - l);
                    const float2 w = mul(wA[p], wr(2 * P3, l));
                    const float2 xa = x[ea], xbv = x[eb];
                    const float2 E = scl(add(xa, conjf2(xbv)), inv2M);
                    const float2 O = scl(mulc(sub(xa, conjf2(xbv)), w), inv2M);
                    const float2 v = f2(-O.y, O.x);
                    x[ea] = add(E, v);
                    x[eb] = conjf2(sub(E, v));
                }
            }
            if (t == 0) {
                // the general formula above paired column 0 with itself wrongly: recompute
                // column 0 (l = 0 packs (X0, XM); pairs l <-> P3 - l) and column 128 (l <-> P3-1-l)
                float2 c0[P3], c1[P3];
#pragma unroll
                for (int l = 0; l < P3; l++) { c0[l] = ld1(j.slot, l); c1[l] = ld1(j.slot, P3 + l); }
                {
                    const float X0 = c0[0].x, XM = c0[0].y;
                    x[0] = f2((X0 + XM) * inv2M, (X0 - XM) * inv2M);
                }
#pragma unroll
                for (int l = 1; l < P3; l++) {
                    if (l <= P3 - l) {
                        const int ea = l, eb = P3 - l;
                        const float2 w = wr(2 * P3, l);
                        const float2 xa = c0[ea], xbv = c0[eb];
                        const float2 E = scl(add(xa, conjf2(xbv)), inv2M);
                        const float2 O = scl(mulc(sub(xa, conjf2(xbv)), w), inv2M);
                        const float2 v = f2(-O.y, O.x);
                        x[ea] = add(E, v);
                        if (eb != ea) x[eb] = conjf2(sub(E, v));
                    }
                }
#pragma unroll
                for (int l = 0; l < P3; l++) {
                    if (l <= P3 - 1 - l) {
                        const int ea = l, eb = P3 - 1 - l;
                        const float2 w = mul(w128, wr(2 * P3, l));
                        const float2 xa = c1[ea], xbv = c1[eb];
                        const float2 E = scl(add(xa, conjf2(xbv)), inv2M);
                        const float2 O = scl(mulc(sub(xa, conjf2(xbv)), w), inv2M);
                        const float2 v = f2(-O.y, O.x);
                        x[P3 + ea] = add(E, v);
                        if (eb != ea) x[P3 + eb] = conjf2(sub(E, v));
                    }
                }
            }
            // stage 3 inverse: per column, P3-point inverse DFT over l_a -> m_a
#pragma unroll
            for (int p = 0; p < Q / 2; p++) {
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    float2 w[P3];
#pragma unroll
                    for (int l = 0; l < P3; l++) w[l] = x[(2 * p + s) * P3 + l];
                    Dft<P3, true>::run(w);
                    const int c = s == 0 ? cA[p] : colB(p);
#pragma unroll
                    for (int m = 0; m < P3; m++) xb[m * 256 + c] = w[m];
                }
            }
        }
        gsync();
        // ---------------- stage 2 (forward) / stage 2 inverse (x is dead here and reused)
        if (j.kind == J_FWD) {
#pragma unroll
            for (int mb = 0; mb < 16; mb++) x[mb] = xb[kb * (T + 1) + ma + P3 * mb];
        } else if (j.kind == J_INV) {
#pragma unroll
            for (int l = 0; l < 16; l++) x[l] = xb[ma * 256 + l * 16 + kb];
        }
        gsync();
        if (j.kind == J_FWD) {
            Dft<16, false>::run(x);
#pragma unroll
            for (int l = 1; l < 16; l++) x[l] = mul(x[l], s_tw2[ma * 16 + l]);
#pragma unroll
            for (int l = 0; l < 16; l++) xb[ma * 256 + l * 16 + kb] = x[l];
        } else if (j.kind == J_INV) {
#pragma unroll
            for (int l = 1; l < 16; l++) x[l] = mulc(x[l], s_tw2[ma * 16 + l]);
            Dft<16, true>::run(x);
#pragma unroll
            for (int mb = 0; mb < 16; mb++) xb[kb * (T + 1) + ma + P3 * mb] = x[mb];
        }
        gsync();
        if (j.kind == J_FWD) {
            // ---------------- stage 3 forward: columns, then pair post-processing
#pragma unroll
            for (int p = 0; p < Q / 2; p++) {
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    const int c = s == 0 ? cA[p] : colB(p);
                    float2 w[P3];
#pragma unroll
                    for (int m = 0; m < P3; m++) w[m] = xb[m * 256 + c];
                    Dft<P3, false>::run(w);
#pragma unroll
                    for (int l = 0; l < P3; l++) x[(2 * p + s) * P3 + l] = w[l];
                }
            }
            float2 z0[P3], z1[P3];                  // column 0 and 128 of thread 0, kept for the fix-up
            if (t == 0) {
#pragma unroll
                for (int l = 0; l < P3; l++) { z0[l] = x[l]; z1[l] = x[P3 + l]; }
            }
            // X[k] = e - u, X[M-k] = conj(e + u), e = (a + conj b)/2, u = (i/2) W_N^k (a - conj b)
#pragma unroll
            for (int p = 0; p < Q / 2; p++) {
#pragma unroll
                for (int l = 0; l < P3; l++) {
                    const int ea = (2 * p) * P3 + l, eb = (2 * p + 1) * P3 + (P3 - 1 - l);
                    const float2 w = mul(wA[p], wr(2 * P3, l));
                    const float2 av = x[ea], bv = x[eb];
                    const float2 e = scl(add(av, conjf2(bv)), 0.5f);
                    const float2 wd = mul(w, sub(av, conjf2(bv)));
                    const float2 u = f2(-0.5f * wd.y, 0.5f * wd.x);
                    x[ea] = sub(e, u);
                    x[eb] = conjf2(add(e, u));
                }
            }
            if (t == 0) {
                x[0] = f2(z0[0].x + z0[0].y, z0[0].x - z0[0].y);     // (X0, X_M) packed
#pragma unroll
                for (int l = 1; l < P3; l++) {
                    if (l <= P3 - l) {
                        const int ea = l, eb = P3 - l;
                        const float2 w = wr(2 * P3, l);
                        const float2 av = z0[ea], bv = z0[eb];
                        const float2 e = scl(add(av, conjf2(bv)), 0.5f);
                        const float2 wd = mul(w, sub(av, conjf2(bv)));
                        const float2 u = f2(-0.5f * wd.y, 0.5f * wd.x);
                        x[ea] = sub(e, u);
                        if (eb != ea) x[eb] = conjf2(add(e, u));
                    }
                }
#pragma unroll
                for (int l = 0; l < P3; l++) {
                    if (l <= P3 - 1 - l) {
                        const int ea = l, eb = P3 - 1 - l;
                        const float2 w = mul(w128, wr(2 * P3, l));
                        const float2 av = z1[ea], bv = z1[eb];
                        const float2 e = scl(add(av, conjf2(bv)), 0.5f);
                        const float2 wd = mul(w, sub(av, conjf2(bv)));
                        const float2 u = f2(-0.5f * wd.y, 0.5f * wd.x);
                        x[P3 + ea] = sub(e, u);
                        if (eb != ea) x[P3 + eb] = conjf2(add(e, u));
                    }
                }
            }
            // ---------------- epilogue: per-mode updates on thread-owned kappa (pairs of elements)
            const int p = j.row;
            const int ds = j.slot;
            const float4* sym = a.sym;
            auto kap_of = [&](int e) {
                const int pp = e / (2 * P3), s = (e / P3) & 1, l = e % P3;
                return (s == 0 ? cA[pp] : colB(pp)) + 256 * l;
            };
            auto lo = [](float4 v) { return f2(v.x, v.y); };
            auto hi = [](float4 v) { return f2(v.z, v.w); };
            switch (j.epi) {
            case X_STORE:
#pragma unroll
                for (int e = 0; e < 16; e += 2) st2(ds, e, x[e], x[e + 1]);
                break;
            case X_B1: {        // B1 -= a2 (E3(p+1) - E3(p))
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    const float4 u = ld2(sE3(p + 1), e), v = ld2(sE3(p), e);
                    st2(ds, e, sub(x[e], scl(sub(lo(u), lo(v)), a2)), sub(x[e + 1], scl(sub(hi(u), hi(v)), a2)));
                }
            } break;
            case X_B2: {        // B2 += S E3(p)
                const float2 e30 = ld1(sE3(p), 0);
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    const float4 qa = sym[kap_of(e)], qb = sym[kap_of(e + 1)];
                    const float4 v = ld2(sE3(p), e);
                    st2(ds, e, add(x[e], mul(f2(qa.x, qa.y), lo(v))), add(x[e + 1], mul(f2(qb.x, qb.y), hi(v))));
                }
                if (t == 0) {                     // packed DC/Nyquist element: two real updates
                    const float sd = sym[0].x, sn = sym[M].x;
                    slots[sidx(ds, 0)] = f2(x[0].x + sd * e30.x, x[0].y + sn * e30.y);
                }
            } break;
            case X_B3: {        // B3 += a2 (E1(p+1) - E1(p)) - S E2(p)
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    const float4 qa = sym[kap_of(e)], qb = sym[kap_of(e + 1)];
                    const float4 u = ld2(sE1(p + 1), e), v = ld2(sE1(p), e), w2 = ld2(sE2, e);
                    st2(ds, e, sub(add(x[e], scl(sub(lo(u), lo(v)), a2)), mul(f2(qa.x, qa.y), lo(w2))),
                        sub(add(x[e + 1], scl(sub(hi(u), hi(v)), a2)), mul(f2(qb.x, qb.y), hi(w2))));
                }
                if (t == 0) {
                    const float sd = sym[0].x, sn = sym[M].x;
                    const float2 d = sub(ld1(sE1(p + 1), 0), ld1(sE1(p), 0)), e2 = ld1(sE2, 0);
                    slots[sidx(ds, 0)] = f2(x[0].x + a2 * d.x - sd * e2.x, x[0].y + a2 * d.y - sn * e2.y);
                }
            } break;
            case X_J1: {        // E1 += a2 (B3(p) - B3(p-1)) - cj1 j1
                float cj1[16];
#pragma unroll
                for (int e = 0; e < 16; e++) cj1[e] = sym[kap_of(e)].z;
                const float cjn = (t == 0) ? sym[M].z : cj1[0];   // Nyquist half of the packed element
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    const float4 u = ld2(sB3(p), e), v = ld2(sB3(p - 1), e), d0 = ld2(ds, e);
                    const float2 da = sub(lo(u), lo(v)), db = sub(hi(u), hi(v));
                    const float cy = (e == 0) ? cjn : cj1[e];
                    st2(ds, e, f2(d0.x + a2 * da.x - cj1[e] * x[e].x, d0.y + a2 * da.y - cy * x[e].y),
                        f2(d0.z + a2 * db.x - cj1[e + 1] * x[e + 1].x, d0.w + a2 * db.y - cj1[e + 1] * x[e + 1].y));
                }
            } break;
            case X_J2: {        // E2 += conj(S) B3(p) - cj j2
                const float2 b30 = ld1(sB3(p), 0), e20 = ld1(ds, 0);
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    const float4 qa = sym[kap_of(e)], qb = sym[kap_of(e + 1)];
                    const float4 u = ld2(sB3(p), e), d0 = ld2(ds, e);
                    const float2 sa = mulc(lo(u), f2(qa.x, qa.y)), sb = mulc(hi(u), f2(qb.x, qb.y));
                    st2(ds, e, f2(d0.x + sa.x - qa.w * x[e].x, d0.y + sa.y - qa.w * x[e].y),
                        f2(d0.z + sb.x - qb.w * x[e + 1].x, d0.w + sb.y - qb.w * x[e + 1].y));
                }
                if (t == 0) {                     // real symbols at DC and Nyquist
                    const float4 qd = sym[0], qn = sym[M];
                    slots[sidx(ds, 0)] = f2(e20.x + qd.x * b30.x - qd.w * x[0].x, e20.y + qn.x * b30.y - qn.w * x[0].y);
                }
            } break;
            default: {          // X_J3: E3 += -conj(S) B2(p) - a2 (B1(p) - B1(p-1)) - cj j3
                const float2 b20 = ld1(sB2, 0), e30 = ld1(ds, 0);
                const float2 dd0 = sub(ld1(sB1(p), 0), ld1(sB1(p - 1), 0));
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    const float4 qa = sym[kap_of(e)], qb = sym[kap_of(e + 1)];
                    const float4 b2 = ld2(sB2, e), u = ld2(sB1(p), e), v = ld2(sB1(p - 1), e), d0 = ld2(ds, e);
                    const float2 sa = mulc(lo(b2), f2(qa.x, qa.y)), sb = mulc(hi(b2), f2(qb.x, qb.y));
                    const float2 da = sub(lo(u), lo(v)), db = sub(hi(u), hi(v));
                    st2(ds, e, f2(d0.x - sa.x - a2 * da.x - qa.w * x[e].x, d0.y - sa.y - a2 * da.y - qa.w * x[e].y),
                        f2(d0.z - sb.x - a2 * db.x - qb.w * x[e + 1].x, d0.w - sb.y - a2 * db.y - qb.w * x[e + 1].y));
                }
                if (t == 0) {
                    const float4 qd = sym[0], qn = sym[M];
                    slots[sidx(ds, 0)] = f2(e30.x - qd.x * b20.x - a2 * dd0.x - qd.w * x[0].x,
                                            e30.y - qn.x * b20.y - a2 * dd0.y - qn.w * x[0].y);
                }
            } break;
            }
        } else if (j.kind == J_INV) {
            // ---------------- stage 1 inverse: gather over k_b, twiddle, 16-point inverse DFT, store
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = xb[k * (T + 1) + t];
#pragma unroll
            for (int k = 1; k < 16; k++) x[k] = mulc(x[k], tw1[k]);
            Dft<16, true>::run(x);
            float2* d = reinterpret_cast<float2*>(j.dst);
#pragma unroll
            for (int nb = 0; nb < 16; nb++) stg_stream(d + t + T * nb, x[nb]);
        }
        if (cta_sync_after(ri)) __syncthreads(); else gsync();
        if (fm && threadIdx.x == 0) {
            if (ri == 0) { __threadfence(); st_release(fb.flags + 2 * strip, fb.epoch); }
            if (ri == 2) st_release(fb.flags + 2 * strip + 1, fb.epoch);
        }
    }
  }
}

// copies the 7 halo rows of every work item: E1,E2,E3,B1,B3 of row p0-1 and E1,E3 of row p1
__global__ void k_halo(FusedBatch fb, int n1, int k0) {
    const int4 it = fb.items[blockIdx.x];
    const FusedInst& a = fb.inst[it.x];
    const int k = k0 + blockIdx.y;
    const int n2 = a.n2, p0 = it.z, p1 = it.w;
    const int rl = (p0 - 1 + n2) % n2, rn = p1 % n2;
    const float* src;
    switch (k) {
    case 0: src = a.E[0] + (size_t)rl * n1; break;
    case 1: src = a.E[1] + (size_t)rl * n1; break;
    case 2: src = a.E[2] + (size_t)rl * n1; break;
    case 3: src = a.B[0] + (size_t)rl * n1; break;
    case 4: src = a.B[2] + (size_t)rl * n1; break;
    case 5: src = a.E[0] + (size_t)rn * n1; break;
    default: src = a.E[2] + (size_t)rn * n1; break;
    }
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(const_cast<float*>(a.halo) + ((size_t)it.y * 7 + k) * n1);
    for (int i = threadIdx.x; i < n1 / 4; i += blockDim.x) d4[i] = s4[i];
}

// ------------------------------------------------------------------ host side
bool fused_supported(const hyb_grid_desc& d) {
    return d.precision == 32 && d.dims == 2 && (d.n1 == 512 || d.n1 == 1024 || d.n1 == 2048 || d.n1 == 4096) && d.n2 >= 4;
}

template <int N>
static size_t fused_smem() { return sizeof(float2) * ((size_t)kSlots * Geo<N>::M + 3 * (size_t)Geo<N>::XB + 16 * Geo<N>::P3); }

size_t fused_smem_bytes(int n1) { return n1 == 4096 ? fused_tm_smem_bytes() : fused_tmt_smem_bytes(n1); }

template <int N>
static cudaError_t fused_attr(int* occ) {
    const size_t smem = fused_smem<N>();
    cudaError_t e = cudaFuncSetAttribute(k_fused2d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_fused2d<N>, Geo<N>::NT, smem);
}

// resident CTAs per SM of the fused kernel for n1
cudaError_t fused_occupancy(int n1, int* occ) { return n1 == 4096 ? fused_tm_occupancy(occ) : fused_tmt_occupancy(n1, occ); }

template <int N>
static cudaError_t launch_n(const FusedBatch& fb, int grid, cudaStream_t s) {
    const size_t smem = fused_smem<N>();
    if (fb.flags) {          // all CTAs must be resident together: cooperative launch
        void* args[] = {const_cast<FusedBatch*>(&fb)};
        return cudaLaunchCooperativeKernel((const void*)k_fused2d<N>, dim3(grid), dim3(Geo<N>::NT), args, smem, s);
    }
    k_fused2d<N><<<grid, Geo<N>::NT, smem, s>>>(fb);
    return cudaGetLastError();
}

// one step for the work items of a launch: halo copy (unless the kernel exchanges
// halos itself), then the persistent fused kernel
cudaError_t halo_parts(int n1, const FusedBatch& fb, int k0, int nk, cudaStream_t s) {
    if (fb.n_items < 1 || nk < 1) return cudaSuccess;
    k_halo<<<dim3(fb.n_items, nk), 256, 0, s>>>(fb, n1, k0);
    return cudaGetLastError();
}

__global__ void k_copy_rows(const RowCopy* __restrict__ tasks) {
    const RowCopy t = tasks[blockIdx.x];
    const float4* s4 = reinterpret_cast<const float4*>(t.src);
    float4* d4 = reinterpret_cast<float4*>(t.dst);
    for (int i = threadIdx.x; i < t.n / 4; i += blockDim.x) d4[i] = s4[i];
}

cudaError_t copy_rows(const RowCopy* tasks, int n, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    k_copy_rows<<<n, 256, 0, s>>>(tasks);
    return cudaGetLastError();
}

cudaError_t fused_kernel_launch(int n1, const FusedBatch& fb, int grid, cudaStream_t s) {
    return n1 == 4096 ? fused_tm_launch(fb, grid, s) : fused_tmt_launch(n1, fb, grid, s);
}

cudaError_t fused_launch(int n1, const FusedBatch& fb, int grid, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    cudaError_t e;
    if (!fb.flags) {
        e = halo_parts(n1, fb, 0, 7, s);
        if (e != cudaSuccess) return e;
    }
    if (ev0) { e = cudaEventRecord(ev0, s); if (e != cudaSuccess) return e; }
    e = fused_kernel_launch(n1, fb, grid, s);
    if (e != cudaSuccess) return e;
    if (ev1) e = cudaEventRecord(ev1, s);
    return e;
}

// per-grid tables of the fused kernel (symbols, W_N^c) and its halo buffer
hyb_status fused_tables(hyb_grid* g, int n_strips, FusedPlan* P) {
    const int N = g->d.n1, M = N / 2;
    std::vector<float2> S(M + 1);
    std::vector<float> cj1(M + 1), cj(M + 1);
    HYB_CUDA_TRY(cudaMemcpy(S.data(), g->tf.S, sizeof(float2) * (M + 1), cudaMemcpyDeviceToHost));
    HYB_CUDA_TRY(cudaMemcpy(cj1.data(), g->tf.cj1, sizeof(float) * (M + 1), cudaMemcpyDeviceToHost));
    HYB_CUDA_TRY(cudaMemcpy(cj.data(), g->tf.cj, sizeof(float) * (M + 1), cudaMemcpyDeviceToHost));
    std::vector<float4> sym(M + 1);
    for (int k = 0; k <= M; k++) sym[k] = make_float4(S[k].x, S[k].y, cj1[k], cj[k]);
    HYB_CUDA_TRY(cudaMalloc(&P->sym, sizeof(float4) * (M + 1)));
    HYB_CUDA_TRY(cudaMemcpy(P->sym, sym.data(), sizeof(float4) * (M + 1), cudaMemcpyHostToDevice));
    std::vector<float2> twC(256);
    const double pi = 3.14159265358979323846;
    for (int c = 0; c < 256; c++) { const double ang = -2.0 * pi * c / N; twC[c] = make_float2((float)cos(ang), (float)sin(ang)); }
    HYB_CUDA_TRY(cudaMalloc(&P->twC, sizeof(float2) * 256));
    HYB_CUDA_TRY(cudaMemcpy(P->twC, twC.data(), sizeof(float2) * 256, cudaMemcpyHostToDevice));
    P->twM = g->tf.twM;
    HYB_CUDA_TRY(cudaMalloc(&P->halo, sizeof(float) * (size_t)n_strips * 7 * N));
    P->n_strips = n_strips;
    return HYB_OK;
}

// re-plans a fused grid for n_strips strips (halo buffer and single-grid items)
hyb_status fused_set_strips(hyb_grid* g, int n_strips) {
    FusedPlan* P = g->fused;
    if (n_strips < 1) n_strips = 1;
    if (n_strips > g->d.n2) n_strips = g->d.n2;
    if (P->halo) { cudaFree(P->halo); P->halo = nullptr; }
    HYB_CUDA_TRY(cudaMalloc(&P->halo, sizeof(float) * (size_t)n_strips * 7 * g->d.n1));
    P->n_strips = n_strips;
    std::vector<int4> it = fused_items(0, g->d.n2, n_strips);
    if (P->items) { cudaFree(P->items); P->items = nullptr; }
    HYB_CUDA_TRY(cudaMalloc(&P->items, sizeof(int4) * it.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->items, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    P->n_items = (int)it.size();
    int occ = 0, sms = 0;
    HYB_CUDA_TRY(fused_occupancy(g->d.n1, &occ));
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    P->grid = P->n_items < sms * occ ? P->n_items : sms * occ;
    if (P->flags) { cudaFree(P->flags); P->flags = nullptr; }
    if (P->n_items <= sms * occ && fused_in_kernel_halo(g->d.n1)) {
        HYB_CUDA_TRY(cudaMalloc(&P->flags, sizeof(int) * 2 * (size_t)n_strips));
        HYB_CUDA_TRY(cudaMemset(P->flags, 0, sizeof(int) * 2 * (size_t)n_strips));
        P->epoch = 0;
    }
    return HYB_OK;
}

// rows split into n_strips nearly equal strips: items {inst, strip, p0, p1}
std::vector<int4> fused_items(int inst, int n2, int n_strips) {
    std::vector<int4> it(n_strips);
    for (int s = 0; s < n_strips; s++)
        it[s] = make_int4(inst, s, (int)(((int64_t)s * n2) / n_strips), (int)(((int64_t)(s + 1) * n2) / n_strips));
    return it;
}

FusedInst fused_inst(const hyb_grid* g) {
    FusedInst a;
    const FusedPlan* P = g->fused;
    for (int c = 0; c < 3; c++) { a.E[c] = (float*)g->E[c]; a.B[c] = (float*)g->B[c]; a.J[c] = (const float*)g->J[c]; }
    a.halo = P->halo;
    a.sym = P->sym;
    a.twM = P->twM;
    a.twC = P->twC;
    a.a2 = (float)(g->d.dt / g->d.dx2);
    a.n2 = g->d.n2;
    return a;
}

// The halo rows of a single grid's strips are exchanged inside the kernel (one co-resident
// CTA per strip, cooperative launch) for n1 = 4096.  The n1 = 512 .. 2048 kernel runs two CTAs
// per SM, which the runtime's cooperative launch does not admit (it counts one per SM), so those
// grids copy their halo rows in a small launch before the step instead.
bool fused_in_kernel_halo(int n1) { return n1 == 4096; }

hyb_status fused_create(hyb_grid* g) {
    FusedPlan* P = new FusedPlan();
    g->fused = P;
    int occ = 0, sms = 0;
    HYB_CUDA_TRY(fused_occupancy(g->d.n1, &occ));
    if (occ < 1) { set_error("fused kernel does not fit on an SM"); return HYB_EINVAL; }
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    int ns = sms * occ;
    if (ns > g->d.n2 / 2) ns = g->d.n2 / 2;
    if (ns < 1) ns = 1;
    hyb_status st = fused_tables(g, ns, P);
    if (st != HYB_OK) return st;
    std::vector<int4> it = fused_items(0, g->d.n2, ns);
    HYB_CUDA_TRY(cudaMalloc(&P->items, sizeof(int4) * it.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->items, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    P->n_items = (int)it.size();
    P->grid = (int)it.size();
    if (fused_in_kernel_halo(g->d.n1)) {
        HYB_CUDA_TRY(cudaMalloc(&P->flags, sizeof(int) * 2 * (size_t)ns));
        HYB_CUDA_TRY(cudaMemset(P->flags, 0, sizeof(int) * 2 * (size_t)ns));
    }
    P->epoch = 0;
    return HYB_OK;
}

static void hp_release(FusedPlan* P) {
    if (P->hp_items) cudaFree(P->hp_items);
    if (P->hp_halo) cudaFree(P->hp_halo);
    for (cudaStream_t& q : P->hp_s) { if (q) cudaStreamDestroy(q); q = nullptr; }
    for (cudaEvent_t e : P->hp_ev) if (e) cudaEventDestroy(e);
    P->hp_items = nullptr;
    P->hp_halo = nullptr;
    P->hp_ev.clear();
    P->hp_chunks = 0;
}

void fused_destroy(hyb_grid* g) {
    FusedPlan* P = g->fused;
    if (!P) return;
    hp_release(P);
    if (P->items) cudaFree(P->items);
    if (P->halo) cudaFree(P->halo);
    if (P->flags) cudaFree(P->flags);
    if (P->sym) cudaFree(P->sym);
    if (P->twC) cudaFree(P->twC);
    delete P;
    g->fused = nullptr;
}

hyb_status fused_advance(hyb_grid* g, int nsteps) {
    FusedPlan* P = g->fused;
    FusedBatch fb;
    fb.inst[0] = fused_inst(g);
    fb.items = P->items;
    fb.n_items = P->n_items;
    fb.flags = P->flags;          // in-kernel halo exchange: one co-resident CTA per strip
    fb.n_strips = P->n_strips;
    fb.err = g->dflag;
    for (int s = 0; s < nsteps; s++) {
        fb.epoch = ++P->epoch;
        HYB_CUDA_TRY(fused_launch(g->d.n1, fb, P->grid, g->stream, g->ev_start, g->ev_stop));
    }
    return HYB_OK;
}

int fused_launches_per_step(const hyb_grid* g) { return (g->fused && g->fused->flags) ? 1 : 2; }

const char* fused_step_kernel(const hyb_grid* g) {
    switch (g->d.n1) {
    case 512: return "k_fused_tmt<32>";
    case 1024: return "k_fused_tmt<64>";
    case 2048: return "k_fused_tmt<128>";
    default: return "k_fused_tm";
    }
}

// ------------------------------------------------------------------ one step from and to host arrays
// The copies over the host link dominate this step, so it is pipelined over chunks of rows:
// stream 0 copies the rows in (the last row first, then chunk by chunk), stream 1 fills the
// halo buffer and runs the fused kernel on chunk c as soon as chunks c and c + 1 have landed,
// stream 2 copies chunk c's E and B back once it is computed, while later chunks still come in.
// Halo rows must be taken before the rows they come from are updated in place: the lower
// parts of chunk c + 1 (row p0 - 1 of its strips, the first of which is the last row of chunk
// c) before chunk c runs, and the upper part of the very last strip (row 0) before chunk 0 runs.
static hyb_status hp_plan(hyb_grid* g) {
    FusedPlan* P = g->fused;
    if (P->hp_chunks) return HYB_OK;
    hp_release(P);                                 // whatever an earlier, failed plan left
    const int n2 = g->d.n2;
    const int C = std::max(1, std::min(4, n2 / 8));
    std::vector<int4> items;
    P->hp_first.assign(1, 0);
    P->hp_row0.assign(1, 0);
    for (int c = 0; c < C; c++) {
        const int r0 = (int)((int64_t)c * n2 / C), r1 = (int)((int64_t)(c + 1) * n2 / C);
        const int ns = std::max(1, (r1 - r0) / 2);
        for (int s = 0; s < ns; s++) {
            const int p0 = r0 + (int)((int64_t)s * (r1 - r0) / ns), p1 = r0 + (int)((int64_t)(s + 1) * (r1 - r0) / ns);
            items.push_back(make_int4(0, (int)items.size(), p0, p1));
        }
        P->hp_first.push_back((int)items.size());
        P->hp_row0.push_back(r1);
    }
    HYB_CUDA_TRY(cudaMalloc(&P->hp_items, sizeof(int4) * items.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->hp_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMalloc(&P->hp_halo, sizeof(float) * items.size() * 7 * (size_t)g->d.n1));
    for (auto& q : P->hp_s) HYB_CUDA_TRY(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    P->hp_ev.assign(2 + 2 * (size_t)C, nullptr);
    for (auto& e : P->hp_ev) HYB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    P->hp_chunks = C;
    return HYB_OK;
}

hyb_status fused_host_advance(hyb_grid* g, void* const E[3], void* const B[3], void* const J[3]) {
    hyb_status st = hp_plan(g);
    if (st != HYB_OK) return st;
    FusedPlan* P = g->fused;
    const int n1 = g->d.n1, n2 = g->d.n2, C = P->hp_chunks;
    const size_t rowb = sizeof(float) * (size_t)n1;
    cudaStream_t in = P->hp_s[0], cmp = P->hp_s[1], out = P->hp_s[2];
    cudaEvent_t fork = P->hp_ev[0], join = P->hp_ev[1];
    auto ev_in = [&](int c) { return P->hp_ev[2 + c]; };
    auto ev_cmp = [&](int c) { return P->hp_ev[2 + C + c]; };
    void* const* hf[3] = {E, B, J};
    void* df[3][3];
    for (int c = 0; c < 3; c++) { df[0][c] = g->E[c]; df[1][c] = g->B[c]; df[2][c] = g->J[c]; }
    auto rows_copy = [&](int kind, int comp, int r0, int r1, cudaMemcpyKind dir, cudaStream_t s) {
        char* d = (char*)df[kind][comp] + (size_t)r0 * rowb;
        char* h = (char*)hf[kind][comp] + (size_t)r0 * rowb;
        return dir == cudaMemcpyHostToDevice ? cudaMemcpyAsync(d, h, (size_t)(r1 - r0) * rowb, dir, s)
                                             : cudaMemcpyAsync(h, d, (size_t)(r1 - r0) * rowb, dir, s);
    };
    FusedBatch fb;
    fb.inst[0] = fused_inst(g);
    fb.inst[0].halo = P->hp_halo;
    fb.flags = nullptr;
    fb.epoch = 0;
    fb.n_strips = 0;
    fb.err = g->dflag;
    auto sub = [&](int i0, int i1) {
        FusedBatch b = fb;
        b.items = P->hp_items + i0;
        b.n_items = i1 - i0;
        return b;
    };
    int occ = 0, sms = 0;
    HYB_CUDA_TRY(fused_occupancy(n1, &occ));
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    const int last = P->hp_first[C] - 1;                   // the strip that ends at row n2 (wraps to row 0)
    // chunk ch's rows of all nine arrays, plus the first row of chunk ch + 1 for E1 and E3 (the
    // upper halo of the chunk's last strip), so that compute ch waits for its own copy only
    auto copy_in = [&](int ch) -> cudaError_t {
        for (int k = 0; k < 3; k++)
            for (int c = 0; c < 3; c++) {
                const int extra = (k == 0 && c != 1 && ch + 1 < C) ? 1 : 0;
                cudaError_t e = rows_copy(k, c, P->hp_row0[ch], P->hp_row0[ch + 1] + extra, cudaMemcpyHostToDevice, in);
                if (e != cudaSuccess) return e;
            }
        return cudaEventRecord(ev_in(ch), in);
    };
    HYB_CUDA_TRY(cudaEventRecord(fork, g->stream));
    for (cudaStream_t q : P->hp_s) HYB_CUDA_TRY(cudaStreamWaitEvent(q, fork, 0));
    // the copy-in stream runs ahead chunk by chunk; compute ch waits for copy ch, copy-out ch for compute ch.
    // Halo rows are taken into the halo buffer before the chunk that holds them is updated.
    for (int k = 0; k < 3; k++)
        for (int c = 0; c < 3; c++) HYB_CUDA_TRY(rows_copy(k, c, n2 - 1, n2, cudaMemcpyHostToDevice, in));
    HYB_CUDA_TRY(copy_in(0));
    HYB_CUDA_TRY(cudaStreamWaitEvent(cmp, ev_in(0), 0));
    HYB_CUDA_TRY(halo_parts(n1, sub(last, last + 1), 5, 2, cmp));          // row 0, before chunk 0 runs
    HYB_CUDA_TRY(halo_parts(n1, sub(P->hp_first[0], P->hp_first[1]), 0, 5, cmp));
    for (int ch = 0; ch < C; ch++) {
        if (ch + 1 < C) HYB_CUDA_TRY(copy_in(ch + 1));
        const int i0 = P->hp_first[ch], i1 = P->hp_first[ch + 1];
        if (ch > 0) {
            HYB_CUDA_TRY(cudaStreamWaitEvent(cmp, ev_in(ch), 0));
            HYB_CUDA_TRY(halo_parts(n1, sub(i0 + 1, i1), 0, 5, cmp));      // lower halos inside chunk ch
        }
        HYB_CUDA_TRY(halo_parts(n1, sub(i0, ch + 1 == C ? i1 - 1 : i1), 5, 2, cmp));
        if (ch + 1 < C) HYB_CUDA_TRY(halo_parts(n1, sub(i1, i1 + 1), 0, 5, cmp));   // row r1 - 1, for chunk ch + 1
        const FusedBatch b = sub(i0, i1);
        HYB_CUDA_TRY(fused_kernel_launch(n1, b, std::min(b.n_items, sms * occ), cmp));
        HYB_CUDA_TRY(cudaEventRecord(ev_cmp(ch), cmp));
        HYB_CUDA_TRY(cudaStreamWaitEvent(out, ev_cmp(ch), 0));
        for (int k = 0; k < 2; k++)
            for (int c = 0; c < 3; c++) HYB_CUDA_TRY(rows_copy(k, c, P->hp_row0[ch], P->hp_row0[ch + 1], cudaMemcpyDeviceToHost, out));
    }
    HYB_CUDA_TRY(cudaEventRecord(join, out));
    HYB_CUDA_TRY(cudaStreamWaitEvent(g->stream, join, 0));
    return HYB_OK;
}

}  // namespace hyb
