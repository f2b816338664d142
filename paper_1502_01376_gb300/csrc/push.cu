// push.cu -- field gather and relativistic Boris push of the particles.
// Gather: momentum-conserving interpolation (Appendix: every field component is
// interpolated with the order-l shape s_l along each axis, from its own staggered
// grid): F_c(x) = sum_i F_c[i] prod_a S_l(x_a - i_a - sigma_{c,a}), with sigma = 1/2
// along the axes where the component sits at half points (2D: E1 (1/2,0), E2 (0,1/2),
// E3 (0,0), B1 (0,1/2), B2 (1/2,0), B3 (1/2,1/2); 3D: E1 (1/2,0,0), E2 (0,1/2,0),
// E3 (0,0,1/2), B1 (0,1/2,1/2), B2 (1/2,0,1/2), B3 (1/2,1/2,0)).  S_l is the centred
// B-spline of order l; only its l + 1 non-zero points are visited, their weights
// from the spline's pieces without a branch.
// Push (c = 1, u = gamma v): u- = u + h E, t = h B / gamma(u-), s = 2 t / (1 + t.t),
// u' = u- + u- x t, u+ = u- + u' x s, u_new = u+ + h E with h = (q/m) dt / 2, then
// x_new = x + dt u_new / gamma(u_new).  One thread per particle.
#include <climits>

#include "hyb_internal.cuh"

namespace hyb {

// weights of the l + 1 grid points i0 .. i0 + l (relative to the cell) that can be non-zero for a
// particle at offset p from the component's own grid: the pieces of the B-spline written for the
// distance delta to the reference point (l = 1, 3: delta = p - floor(p) in [0, 1); l = 2: delta =
// p - round(p) in [-1/2, 1/2]), so that no branch picks the piece
template <int L, typename T>
__device__ __forceinline__ int pweights(T p, T (&w)[L + 1]) {
    if (L == 1) {
        const T f = floor(p), d = p - f;
        w[0] = (T)1 - d;
        w[1] = d;
        return (int)f;
    }
    if (L == 2) {
        const T f = floor(p + (T)0.5), d = p - f;
        const T a = (T)0.5 - d, b = (T)0.5 + d;
        w[0] = (T)0.5 * a * a;
        w[1] = (T)0.75 - d * d;
        w[2] = (T)0.5 * b * b;
        return (int)f - 1;
    }
    const T f = floor(p), d = p - f, e = (T)1 - d;
    const T d2 = d * d, e2 = e * e;
    w[0] = e2 * e * ((T)1 / (T)6);
    w[1] = ((T)4 - (T)6 * d2 + (T)3 * d2 * d) * ((T)1 / (T)6);
    w[2] = ((T)4 - (T)6 * e2 + (T)3 * e2 * e) * ((T)1 / (T)6);
    w[3] = d2 * d * ((T)1 / (T)6);
    return (int)f - 1;
}

// 1 / sqrt(x): the hardware reciprocal square root in FP32, the rounded quotient in FP64
__device__ __forceinline__ float prsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double prsqrt(double x) { return 1.0 / sqrt(x); }

// periodic index: one add or subtract for the stencil's range (-n <= i < 2n), a modulo only
// for grids narrower than the stencil
__device__ __forceinline__ int pwrap(int i, int n) {
    i = i < 0 ? i + n : i;
    i = i >= n ? i - n : i;
    if ((unsigned)i >= (unsigned)n) i = ((i % n) + n) % n;
    return i;
}

// moves a particle to the cell that holds it (offsets in [-1, 2) on entry); the decision and the new
// offset are taken in T, so that off ends in [0, 1)
template <typename T>
__device__ __forceinline__ bool renormalise(int& c, T& o, int n) {
    if (!(o >= (T)-1 && o < (T)2)) return false;
    if (o < (T)0) { o += (T)1; c -= 1; }
    else if (o >= (T)1) { o -= (T)1; c += 1; }
    if (o >= (T)1) { o = (T)0; c += 1; }          // o = -tiny rounded up to 1
    c = pwrap(c, n);
    return true;
}

template <typename T>
__device__ __forceinline__ void boris(T (&u)[3], const T (&E)[3], const T (&B)[3], T h) {
    T um[3], t[3], up[3], s[3];
#pragma unroll
    for (int a = 0; a < 3; a++) um[a] = u[a] + h * E[a];
    const T gi = prsqrt((T)1 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
    for (int a = 0; a < 3; a++) t[a] = h * B[a] * gi;
    const T f = (T)2 / ((T)1 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
#pragma unroll
    for (int a = 0; a < 3; a++) s[a] = f * t[a];
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    T uq[3];
    uq[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    uq[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    uq[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
#pragma unroll
    for (int a = 0; a < 3; a++) u[a] = uq[a] + h * E[a];
}

struct PushFields { const void* E[3]; const void* B[3]; };

// The block's particles are usually neighbours (a PIC code keeps them sorted by cell): the block
// takes the bounding box of their cells, and when the box widened by the stencil reach (2 points
// each side, every order and staggering) fits the shared tile, it stages the six components there
// with row-contiguous loads and gathers from the tile; otherwise every particle gathers from global
// memory.  Both paths take the same weights and points.
constexpr int kPushThreads = 256;
constexpr int kReach = 2;

template <typename T, int L>
__global__ void __launch_bounds__(kPushThreads, 3) k_push2d(PushFields F, int n1, int n2, int32_t* __restrict__ cell,
                                                          T* __restrict__ off, T* __restrict__ u, const T* __restrict__ qm,
                                                          T* __restrict__ off_new, T* __restrict__ v3, int64_t np, T hdt,
                                                          T s1, T s2, int* __restrict__ flag) {
    constexpr int kTile = sizeof(T) == 4 ? 1024 : 512;        // points per component in the shared tile
    __shared__ T tile[6][kTile];
    __shared__ int red[kPushThreads / 32][4];
    const T* src[6] = {(const T*)F.E[0], (const T*)F.E[1], (const T*)F.E[2],
                       (const T*)F.B[0], (const T*)F.B[1], (const T*)F.B[2]};
    using V2 = cplx<T>;                      // a particle's two offsets, one 8- or 16-byte access
    const int64_t stride = (int64_t)gridDim.x * kPushThreads;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the next particle's cell and offsets are loaded while this one is gathered and pushed
    int2 ncc = make_int2(0, 0);
    V2 noo;
    noo.x = noo.y = (T)0;
    {
        const int64_t p = blockIdx.x * (int64_t)kPushThreads + threadIdx.x;
        if (p < np) { ncc = reinterpret_cast<const int2*>(cell)[p]; noo = reinterpret_cast<const V2*>(off)[p]; }
    }
    for (int64_t base = blockIdx.x * (int64_t)kPushThreads; base < np; base += stride) {
        const int64_t p = base + threadIdx.x;
        const bool live = p < np;
        const int2 cc = ncc;
        const V2 oo = noo;
        if (p + stride < np) {
            ncc = reinterpret_cast<const int2*>(cell)[p + stride];
            noo = reinterpret_cast<const V2*>(off)[p + stride];
        }
        int cx = cc.x, cy = cc.y;
        T ox = oo.x, oy = oo.y;
        const bool ok = live && cx >= 0 && cx < n1 && cy >= 0 && cy < n2 && renormalise(cx, ox, n1) &&
                        renormalise(cy, oy, n2);
        if (live && !ok) {
            atomicOr(flag, 1);
            reinterpret_cast<V2*>(off_new)[p] = oo;
            if (v3) v3[p] = (T)0;
        }
        // bounding box of the block's cells
        int bx0 = __reduce_min_sync(0xffffffffu, ok ? cx : INT_MAX), bx1 = __reduce_max_sync(0xffffffffu, ok ? cx : INT_MIN);
        int by0 = __reduce_min_sync(0xffffffffu, ok ? cy : INT_MAX), by1 = __reduce_max_sync(0xffffffffu, ok ? cy : INT_MIN);
        if (lane == 0) { red[warp][0] = bx0; red[warp][1] = bx1; red[warp][2] = by0; red[warp][3] = by1; }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kPushThreads / 32; w++) {
            bx0 = min(bx0, red[w][0]); bx1 = max(bx1, red[w][1]);
            by0 = min(by0, red[w][2]); by1 = max(by1, red[w][3]);
        }
        const bool any = bx0 <= bx1;
        const int W = any ? bx1 - bx0 + 1 + 2 * kReach : 0, H = any ? by1 - by0 + 1 + 2 * kReach : 0;
        const bool tiled = any && W <= kTile && H <= kTile && W * H <= kTile;
        const int tx0 = bx0 - kReach, ty0 = by0 - kReach;
        if (tiled) {
            for (int q = threadIdx.x; q < W * H; q += kPushThreads) {
                const int yy = q / W, xx = q - yy * W;
                const int64_t gq = (int64_t)pwrap(ty0 + yy, n2) * n1 + pwrap(tx0 + xx, n1);
#pragma unroll
                for (int f = 0; f < 6; f++) tile[f][q] = __ldg(src[f] + gq);
            }
        }
        __syncthreads();
        if (ok) {
            T uu[3] = {u[3 * p], u[3 * p + 1], u[3 * p + 2]};
            // weights for the integer (0) and half (1) positions along each axis
            T wx[2][L + 1], wy[2][L + 1];
            const int ix0 = pweights<L>(ox, wx[0]), ix1 = pweights<L>(ox - (T)0.5, wx[1]);
            const int iy0 = pweights<L>(oy, wy[0]), iy1 = pweights<L>(oy - (T)0.5, wy[1]);
            T e1 = 0, e2 = 0, e3 = 0, b1 = 0, b2 = 0, b3 = 0;
            if (tiled) {
                const int lx = cx - tx0, ly = cy - ty0;
#pragma unroll
                for (int j = 0; j <= L; j++) {
                    const int r0 = (ly + iy0 + j) * W + lx, r1 = (ly + iy1 + j) * W + lx;
                    T a10 = 0, a01 = 0, a00 = 0, b01 = 0, b10 = 0, b11 = 0;
#pragma unroll
                    for (int i = 0; i <= L; i++) {
                        a10 += wx[1][i] * tile[0][r0 + ix1 + i];     // E1 at (1/2, 0)
                        b10 += wx[1][i] * tile[4][r0 + ix1 + i];     // B2 at (1/2, 0)
                        a01 += wx[0][i] * tile[1][r1 + ix0 + i];     // E2 at (0, 1/2)
                        b01 += wx[0][i] * tile[3][r1 + ix0 + i];     // B1 at (0, 1/2)
                        a00 += wx[0][i] * tile[2][r0 + ix0 + i];     // E3 at (0, 0)
                        b11 += wx[1][i] * tile[5][r1 + ix1 + i];     // B3 at (1/2, 1/2)
                    }
                    e1 += wy[0][j] * a10; b2 += wy[0][j] * b10; e3 += wy[0][j] * a00;
                    e2 += wy[1][j] * a01; b1 += wy[1][j] * b01; b3 += wy[1][j] * b11;
                }
            } else {
                int cx0[L + 1], cx1[L + 1];
#pragma unroll
                for (int k = 0; k <= L; k++) { cx0[k] = pwrap(cx + ix0 + k, n1); cx1[k] = pwrap(cx + ix1 + k, n1); }
#pragma unroll
                for (int j = 0; j <= L; j++) {
                    const int64_t r0 = (int64_t)pwrap(cy + iy0 + j, n2) * n1, r1 = (int64_t)pwrap(cy + iy1 + j, n2) * n1;
                    T a10 = 0, a01 = 0, a00 = 0, b01 = 0, b10 = 0, b11 = 0;
#pragma unroll
                    for (int i = 0; i <= L; i++) {
                        a10 += wx[1][i] * __ldg(src[0] + r0 + cx1[i]);
                        b10 += wx[1][i] * __ldg(src[4] + r0 + cx1[i]);
                        a01 += wx[0][i] * __ldg(src[1] + r1 + cx0[i]);
                        b01 += wx[0][i] * __ldg(src[3] + r1 + cx0[i]);
                        a00 += wx[0][i] * __ldg(src[2] + r0 + cx0[i]);
                        b11 += wx[1][i] * __ldg(src[5] + r1 + cx1[i]);
                    }
                    e1 += wy[0][j] * a10; b2 += wy[0][j] * b10; e3 += wy[0][j] * a00;
                    e2 += wy[1][j] * a01; b1 += wy[1][j] * b01; b3 += wy[1][j] * b11;
                }
            }
            const T Ev[3] = {e1, e2, e3}, Bv[3] = {b1, b2, b3};
            boris(uu, Ev, Bv, hdt * qm[p]);
            const T gi = prsqrt((T)1 + uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
            reinterpret_cast<int2*>(cell)[p] = make_int2(cx, cy);
            V2 on;
            on.x = ox; on.y = oy;
            reinterpret_cast<V2*>(off)[p] = on;
            u[3 * p] = uu[0]; u[3 * p + 1] = uu[1]; u[3 * p + 2] = uu[2];
            on.x = ox + s1 * uu[0] * gi;
            on.y = oy + s2 * uu[1] * gi;
            reinterpret_cast<V2*>(off_new)[p] = on;
            if (v3) v3[p] = uu[2] * gi;
        }
        __syncthreads();                     // the tile has been read before the next one is staged
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(256) k_push3d(PushFields F, int n1, int n2, int n3, int32_t* __restrict__ cell,
                                               T* __restrict__ off, T* __restrict__ u, const T* __restrict__ qm,
                                               T* __restrict__ off_new, int64_t np, T hdt, T s1, T s2, T s3,
                                               int* __restrict__ flag) {
    // staggering of E1, E2, E3, B1, B2, B3 along x1, x2, x3 (1 = half point)
    constexpr int sg[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
    const int n[3] = {n1, n2, n3};
    const T sc[3] = {s1, s2, s3};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        T o[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            c[a] = cell[3 * p + a];
            o[a] = off[3 * p + a];
            ok = ok && c[a] >= 0 && c[a] < n[a];
        }
#pragma unroll
        for (int a = 0; a < 3; a++) ok = ok && renormalise(c[a], o[a], n[a]);
        if (!ok) {
            atomicOr(flag, 1);
#pragma unroll
            for (int a = 0; a < 3; a++) off_new[3 * p + a] = off[3 * p + a];
            continue;
        }
        T w[3][2][L + 1];
        int i0[3][2];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            i0[a][0] = pweights<L>(o[a], w[a][0]);
            i0[a][1] = pweights<L>(o[a] - (T)0.5, w[a][1]);
        }
        T fv[6];
#pragma unroll
        for (int f = 0; f < 6; f++) {
            const T* A = (const T*)(f < 3 ? F.E[f] : F.B[f - 3]);
            const int h1 = sg[f][0], h2 = sg[f][1], h3 = sg[f][2];
            T acc = 0;
#pragma unroll
            for (int k = 0; k <= L; k++) {
                const int64_t pk = (int64_t)pwrap(c[2] + i0[2][h3] + k, n3) * n2;
#pragma unroll
                for (int j = 0; j <= L; j++) {
                    const int64_t row = (pk + pwrap(c[1] + i0[1][h2] + j, n2)) * n1;
                    T r = 0;
#pragma unroll
                    for (int i = 0; i <= L; i++) r += w[0][h1][i] * __ldg(A + row + pwrap(c[0] + i0[0][h1] + i, n1));
                    acc += w[2][h3][k] * w[1][h2][j] * r;
                }
            }
            fv[f] = acc;
        }
        T uu[3] = {u[3 * p], u[3 * p + 1], u[3 * p + 2]};
        const T Ev[3] = {fv[0], fv[1], fv[2]}, Bv[3] = {fv[3], fv[4], fv[5]};
        boris(uu, Ev, Bv, hdt * qm[p]);
        const T gi = prsqrt((T)1 + uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cell[3 * p + a] = c[a];
            off[3 * p + a] = o[a];
            u[3 * p + a] = uu[a];
            off_new[3 * p + a] = o[a] + sc[a] * uu[a] * gi;
        }
    }
}

template <typename T>
hyb_status push_fields(hyb_grid* g, void* const E[3], void* const B[3], int32_t* cell, T* off, T* u, const T* qm,
                       T* off_new, T* v3, int64_t np, int order) {
    const hyb_grid_desc& d = g->d;
    if (np == 0) return HYB_OK;
    PushFields F;
    for (int c = 0; c < 3; c++) { F.E[c] = E[c]; F.B[c] = B[c]; }
    const int threads = kPushThreads;
    int sms = 0;
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    const int64_t want = (np + threads - 1) / threads;
    const unsigned blocks = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    const T hdt = (T)(0.5 * d.dt);
    const T s1 = (T)(d.dt / d.dx1), s2 = (T)(d.dt / d.dx2), s3 = (T)(d.dt / d.dx3);
    if (d.dims == 2) {
#define HYB_PUSH2(O) k_push2d<T, O><<<blocks, threads, 0, g->stream>>>(F, d.n1, d.n2, cell, off, u, qm, off_new, v3, np, hdt, s1, s2, g->dflag)
        if (order == 1) HYB_PUSH2(1); else if (order == 2) HYB_PUSH2(2); else HYB_PUSH2(3);
#undef HYB_PUSH2
    } else {
#define HYB_PUSH3(O) k_push3d<T, O><<<blocks, threads, 0, g->stream>>>(F, d.n1, d.n2, d.n3, cell, off, u, qm, off_new, np, hdt, s1, s2, s3, g->dflag)
        if (order == 1) HYB_PUSH3(1); else if (order == 2) HYB_PUSH3(2); else HYB_PUSH3(3);
#undef HYB_PUSH3
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

template <typename T>
hyb_status push(hyb_grid* g, int32_t* cell, T* off, T* u, const T* qm, T* off_new, T* v3, int64_t np, int order) {
    return push_fields<T>(g, g->E, g->B, cell, off, u, qm, off_new, v3, np, order);
}

template hyb_status push<float>(hyb_grid*, int32_t*, float*, float*, const float*, float*, float*, int64_t, int);
template hyb_status push<double>(hyb_grid*, int32_t*, double*, double*, const double*, double*, double*, int64_t, int);
template hyb_status push_fields<float>(hyb_grid*, void* const*, void* const*, int32_t*, float*, float*, const float*,
                                       float*, float*, int64_t, int);
template hyb_status push_fields<double>(hyb_grid*, void* const*, void* const*, int32_t*, double*, double*,
                                        const double*, double*, double*, int64_t, int);

}  // namespace hyb
