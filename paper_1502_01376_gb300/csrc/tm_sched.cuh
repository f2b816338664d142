// tm_sched.cuh -- the round schedule and the real-transform helpers shared by the
// TMEM-resident fused kernels (tm_body.cuh for n1 = 4096, tmt_body.cuh for n1 =
// 512 .. 2048): which row each thread group transforms in each round, where its
// forward rows come from, and the even/odd split of the real transform.
#pragma once
#include "fused_dev.cuh"
#include "packed_dev.cuh"
#include "tm_dev.cuh"

namespace hyb {

// ------------------------------------------------------------------ round schedule
// Group g owns component g of E and B: it transforms E_g and B_g, applies the
// update of E_g (Ampere, with j_g) and of B_g (Faraday), and writes both back.
// Rows outside the strip: h = p0 - 1 (from the fields in flag mode, else from the
// halo buffer [E1, E2, E3, B1, B3 of h; E1, E3 of p1]).
//   prologue  P1: g0 E1(p0), g1 E2(h), g2 E3(p0)   P2: g0 E1(h), g2 E3(h)
//             P3: g0 B1(h) (Faraday), g2 B3(h) (Faraday)
//   row p     R1: g0 E1(p+1), g1 E2(p), g2 E3(p+1)   R2: B_g(p), Faraday
//             R3: j_g(p), Ampere into E_g(p)          R4: inverse E_g(p)   R5: inverse B_g(p)
// Every slot is written by one group only, so the three groups synchronise only where
// slots pass between them: after R1 and R2 (and after the prologue rounds).
__device__ __forceinline__ Job tm_job(const FusedInst& a, int N, int p0, int p1, int ri, int g) {
    Job j{J_IDLE, X_STORE, 0, 0, nullptr, nullptr};
    const int h = p0 - 1;
    if (ri < 3) {
        if (ri == 0) { j.kind = J_FWD; j.slot = (g == 0) ? sE1(p0) : (g == 1) ? sE2 : sE3(p0); }
        else if (ri == 1) { if (g != 1) { j.kind = J_FWD; j.slot = (g == 0) ? sE1(h) : sE3(h); } }
        else if (g != 1) { j.kind = J_FWD; j.epi = (g == 0) ? X_B1 : X_B3; j.slot = (g == 0) ? sB1(h) : sB3(h); j.row = h; }
        return j;
    }
    const int r = (ri - 3) % 5, p = p0 + (ri - 3) / 5;
    if (p >= p1) return j;
    j.row = p;
    const int sE = (g == 0) ? sE1(p) : (g == 1) ? sE2 : sE3(p);
    const int sB = (g == 0) ? sB1(p) : (g == 1) ? sB2 : sB3(p);
    if (r == 0) { j.kind = J_FWD; j.slot = (g == 0) ? sE1(p + 1) : (g == 1) ? sE2 : sE3(p + 1); }
    else if (r == 1) { j.kind = J_FWD; j.epi = X_B1 + g; j.slot = sB; }
    else if (r == 2) { j.kind = J_FWD; j.epi = X_J1 + g; j.slot = sE; }
    else { j.kind = J_INV; j.slot = (r == 3) ? sE : sB; j.dst = ((r == 3) ? a.E[g] : a.B[g]) + (size_t)p * N; }
    return j;
}
__device__ __forceinline__ int tm_npro(int g) { return g == 1 ? 1 : 3; }
// source row of the idx-th forward transform of group g in a work item; *direct is set
// when it is the next strip's published first row (read with plain loads after the flag)
__device__ __forceinline__ const float* tm_src(const FusedInst& a, int N, int strip, int p0, int p1, int g, int idx,
                                               bool fm, int next, bool* direct) {
    *direct = false;
    const float* halo = a.halo + (size_t)strip * 7 * N;
    if (idx < tm_npro(g)) {
        const int h = (p0 - 1 + a.n2) % a.n2;
        if (g == 1) return fm ? a.E[1] + (size_t)h * N : halo + 1 * N;
        const int c = (g == 0) ? 0 : 2;
        if (idx == 0) return a.E[c] + (size_t)p0 * N;
        if (idx == 1) return fm ? a.E[c] + (size_t)h * N : halo + c * N;
        return fm ? a.B[c] + (size_t)h * N : halo + (g == 0 ? 3 : 4) * N;
    }
    const int q = idx - tm_npro(g);
    const int p = p0 + q / 3, r = q % 3;
    if (p >= p1) return nullptr;
    if (r == 1) return a.B[g] + (size_t)p * N;
    if (r == 2) return a.J[g] + (size_t)p * N;
    if (g == 1) return a.E[1] + (size_t)p * N;
    const int c = (g == 0) ? 0 : 2;
    if (p + 1 < p1) return a.E[c] + (size_t)(p + 1) * N;
    if (fm) { *direct = true; return a.halo + ((size_t)next * 7 + (g == 0 ? 0 : 1)) * N; }
    return halo + (g == 0 ? 5 : 6) * N;
}

// the seven twiddles W^{k}, k = 1..7, of a stage from this thread's TMEM words
__device__ __forceinline__ void tw_tmem(uint32_t ta, float2 (&w)[8]) {
    float r[16];
    tm_ld16(ta, r);
    tm_wait_ld();
#pragma unroll
    for (int k = 1; k < 8; k++) w[k] = f2(r[2 * k - 2], r[2 * k - 1]);
}

// forward split of one pair: X[k] = e - u, X[M-k] = conj(e + u), e = (a + conj b)/2,
// u = (i/2) w (a - conj b), w = W_N^k, a = Z[k], b = Z[M-k].  With
// u' = (-wd.y/2, -wd.x/2), wd = w (a - conj b): X[k] = (e.x - u'.x, e.y + u'.y),
// X[M-k] = (e.x + u'.x, u'.y - e.y).
__device__ __forceinline__ void split_fwd(float2 av, float2 bv, float2 w, float2& xk, float2& xmk) {
    const float2 e = vfma(bv, f2(0.5f, -0.5f), vmul(av, f2(0.5f, 0.5f)));
    const float2 wd = mul(w, vfma(bv, f2(-1.f, 1.f), av));
    const float2 up = f2(-0.5f * wd.y, -0.5f * wd.x);
    xk = vfma(up, f2(-1.f, 1.f), e);
    xmk = vfma(e, f2(1.f, -1.f), up);
}
// inverse split of one pair (with the 1/M of the inverse transform folded in as s = 1/(2M)):
// Z[k] = E + iO, Z[M-k] = conj(E - iO), E = s (X[k] + conj X[M-k]),
// O = conj(w) s (X[k] - conj X[M-k])
__device__ __forceinline__ void split_inv(float2 xa, float2 xbv, float2 w, float s, float2& zk, float2& zmk) {
    const float2 xs = vmul(xa, f2(s, s));
    const float2 E = vfma(xbv, f2(s, -s), xs);
    const float2 O = mulc(vfma(xbv, f2(-s, s), xs), w);
    zk = f2(E.x - O.y, E.y + O.x);
    zmk = f2(E.x + O.y, O.x - E.y);
}

// per-mode updates after a forward transform (Faraday or Ampere, or a plain store), two
// chunks of four modes: x are the real-input coefficients of this thread's 8 modes, tw its
// slot base in TMEM (slot s, chunk c at tw + 16 s + 8 c), ts its symbols (S of elements
// 4c..4c+3 at ts + 8c, cj1 at ts + 16 + 4c, cj at ts + 24 + 4c), symN the Nyquist mode's
// symbols, t0 whether this thread owns the packed DC/Nyquist element
__device__ __forceinline__ void tm_epilogue(const Job& j, const float2 (&x)[8], uint32_t tw, uint32_t ts, const float4* symN,
                                            float a2, bool t0) {
    auto ta = [&](int slot, int chunk) { return tw + (uint32_t)(16 * slot + 8 * chunk); };
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
            float w[8], S[8];
            tm_ld8(ta(sE3(p), c), w);
            tm_ld8(ts + 8 * c, S);
            tm_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float2 r = add(x[e0 + i], mul(f2(S[2 * i], S[2 * i + 1]), f2(w[2 * i], w[2 * i + 1])));
                o[2 * i] = r.x; o[2 * i + 1] = r.y;
            }
            if (c == 0 && t0) {   // packed DC/Nyquist: two real updates
                o[0] = x[0].x + S[0] * w[0];
                o[1] = x[0].y + symN->x * w[1];
            }
        } break;
        case X_B3: {        // B3 += a2 (E1(p+1) - E1(p)) - S E2(p)
            float u[8], w[8], e2[8], S[8];
            tm_ld8(ta(sE1(p + 1), c), u);
            tm_ld8(ta(sE1(p), c), w);
            tm_ld8(ta(sE2, c), e2);
            tm_ld8(ts + 8 * c, S);
            tm_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float2 se = mul(f2(S[2 * i], S[2 * i + 1]), f2(e2[2 * i], e2[2 * i + 1]));
                o[2 * i] = x[e0 + i].x + a2 * (u[2 * i] - w[2 * i]) - se.x;
                o[2 * i + 1] = x[e0 + i].y + a2 * (u[2 * i + 1] - w[2 * i + 1]) - se.y;
            }
            if (c == 0 && t0) {
                o[0] = x[0].x + a2 * (u[0] - w[0]) - S[0] * e2[0];
                o[1] = x[0].y + a2 * (u[1] - w[1]) - symN->x * e2[1];
            }
        } break;
        case X_J1: {        // E1 += a2 (B3(p) - B3(p-1)) - cj1 j1
            float u[8], w[8], d[8], cj1[4];
            tm_ld8(ta(sB3(p), c), u);
            tm_ld8(ta(sB3(p - 1), c), w);
            tm_ld8(ta(ds, c), d);
            tm_ld4(ts + 16 + 4 * c, cj1);
            tm_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; i++) {
                o[2 * i] = d[2 * i] + a2 * (u[2 * i] - w[2 * i]) - cj1[i] * x[e0 + i].x;
                o[2 * i + 1] = d[2 * i + 1] + a2 * (u[2 * i + 1] - w[2 * i + 1]) - cj1[i] * x[e0 + i].y;
            }
            if (c == 0 && t0) o[1] = d[1] + a2 * (u[1] - w[1]) - symN->z * x[0].y;
        } break;
        case X_J2: {        // E2 += conj(S) B3(p) - cj j2
            float u[8], d[8], S[8], cj[4];
            tm_ld8(ta(sB3(p), c), u);
            tm_ld8(ta(ds, c), d);
            tm_ld8(ts + 8 * c, S);
            tm_ld4(ts + 24 + 4 * c, cj);
            tm_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float2 sb = mulc(f2(u[2 * i], u[2 * i + 1]), f2(S[2 * i], S[2 * i + 1]));
                o[2 * i] = d[2 * i] + sb.x - cj[i] * x[e0 + i].x;
                o[2 * i + 1] = d[2 * i + 1] + sb.y - cj[i] * x[e0 + i].y;
            }
            if (c == 0 && t0) {
                const float4 qn = *symN;
                o[0] = d[0] + S[0] * u[0] - cj[0] * x[0].x;
                o[1] = d[1] + qn.x * u[1] - qn.w * x[0].y;
            }
        } break;
        default: {          // X_J3: E3 += -conj(S) B2(p) - a2 (B1(p) - B1(p-1)) - cj j3
            float b2[8], u[8], w[8], d[8], S[8], cj[4];
            tm_ld8(ta(sB2, c), b2);
            tm_ld8(ta(sB1(p), c), u);
            tm_ld8(ta(sB1(p - 1), c), w);
            tm_ld8(ta(ds, c), d);
            tm_ld8(ts + 8 * c, S);
            tm_ld4(ts + 24 + 4 * c, cj);
            tm_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float2 sb = mulc(f2(b2[2 * i], b2[2 * i + 1]), f2(S[2 * i], S[2 * i + 1]));
                o[2 * i] = d[2 * i] - sb.x - a2 * (u[2 * i] - w[2 * i]) - cj[i] * x[e0 + i].x;
                o[2 * i + 1] = d[2 * i + 1] - sb.y - a2 * (u[2 * i + 1] - w[2 * i + 1]) - cj[i] * x[e0 + i].y;
            }
            if (c == 0 && t0) {
                const float4 qn = *symN;
                o[0] = d[0] - S[0] * b2[0] - a2 * (u[0] - w[0]) - cj[0] * x[0].x;
                o[1] = d[1] - qn.x * b2[1] - a2 * (u[1] - w[1]) - qn.w * x[0].y;
            }
        } break;
        }
        tm_st8(ta(ds, c), o);
    }
    tm_wait_st();
}

}  // namespace hyb
