// deposit.cu -- charge-conserving current deposit (Sec. 2.3) of particles that
// move from x^n to x^{n+1} within one step, in Esirkepov's density-
// decomposition form, which satisfies the finite-difference continuity
// equation (Eq. continuity) exactly:
//   2D: W1 = dS1 (S2^0 + S2^1)/2,  W2 = dS2 (S1^0 + S1^1)/2,
//       j1(i+1/2,j) = -q/(dt dx2) sum_{i'<=i} W1(i',j),
//       j2(i,j+1/2) = -q/(dt dx1) sum_{j'<=j} W2(i,j'),
//       j3(i,j) = q v3 [S1^0 S2^0/3 + S1^1 S2^0/6 + S1^0 S2^1/6 + S1^1 S2^1/3] / dV;
//   3D: W1 = dS1 (S2^0 S3^0 + dS2 S3^0/2 + S2^0 dS3/2 + dS2 dS3/3), cyclic for W2, W3,
//       j_a = -q/(dt dV/dx_a) cumulative sum of W_a along axis a.
// S are B-spline shape factors of order 1, 2 or 3 (grid points at integers).
// One thread per particle; contributions are added with atomics.
#include "hyb_internal.cuh"

namespace hyb {

template <int ORDER, typename T>
__device__ __forceinline__ T bspline(T d) {
    T a = d < (T)0 ? -d : d;
    if (ORDER == 1) return a < (T)1 ? (T)1 - a : (T)0;
    if (ORDER == 2) {
        if (a <= (T)0.5) return (T)0.75 - a * a;
        if (a < (T)1.5) { T t = (T)1.5 - a; return (T)0.5 * t * t; }
        return (T)0;
    }
    if (a <= (T)1) return ((T)4 - (T)6 * a * a + (T)3 * a * a * a) * ((T)1 / (T)6);
    if (a < (T)2) { T t = (T)2 - a; return t * t * t * ((T)1 / (T)6); }
    return (T)0;
}

template <int ORDER> struct Win { static constexpr int lo = (ORDER == 1) ? -1 : -2; static constexpr int n = (ORDER == 1) ? 4 : 6; };

__device__ __forceinline__ int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

// 2D: lanes take particles 8 apart within each chunk of 256, so that for a sorted chunk the
// lanes of a warp sit in different (mostly consecutive) cells and their atomic adds at the same
// window offset go to different, neighbouring addresses.  (A variant that accumulated each block's
// currents in a shared tile first and added each tile point once ran slower: 6.4 against 5.6 ms
// for the 67 M particles of the drifting plasma.)
constexpr int kDepThreads = 256;

template <typename T, int ORDER>
__global__ void __launch_bounds__(kDepThreads) k_deposit2d(T* __restrict__ J1, T* __restrict__ J2, T* __restrict__ J3,
                                                          int n1, int n2, const int32_t* __restrict__ cell,
                                                          const T* __restrict__ off0, const T* __restrict__ off1,
                                                          const T* __restrict__ v3, const T* __restrict__ q, int64_t np,
                                                          T c1s, T c2s, T c3s, int* __restrict__ flag) {
    constexpr int W = Win<ORDER>::n, LO = Win<ORDER>::lo;
    T* const Jc[3] = {J1, J2, J3};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = blockIdx.x * (int64_t)kDepThreads; base < np; base += (int64_t)gridDim.x * kDepThreads) {
        const int64_t p = base + lane * (kDepThreads / 32) + warp;
        if (p >= np) continue;
        const int cx = cell[2 * p], cy = cell[2 * p + 1];
        const T x0 = off0[2 * p], y0 = off0[2 * p + 1], x1 = off1[2 * p], y1 = off1[2 * p + 1];
        const T dx = x1 - x0, dy = y1 - y0;
        if (!(x0 >= (T)0 && x0 < (T)1 && y0 >= (T)0 && y0 < (T)1 && dx > (T)-1 && dx < (T)1 && dy > (T)-1 && dy < (T)1) ||
            cx < 0 || cx >= n1 || cy < 0 || cy >= n2) {
            atomicOr(flag, 1);
            continue;
        }
        // along each axis only the points where the shape at x^n or at x^{n+1} is non-zero: at most
        // ORDER + 2 consecutive points (|x^{n+1} - x^n| < 1 cell), starting at gx, gy (relative to the
        // cell, clamped into the full window LO .. LO + W - 1, which at a rounding edge only drops a
        // point of weight 0); beyond them the cumulative sums are back to 0
        constexpr int WN = ORDER + 2;
        const int gx = min(max((int)floor((x0 < x1 ? x0 : x1) - (T)0.5 * (T)(ORDER + 1)) + 1, LO), LO + W - WN);
        const int gy = min(max((int)floor((y0 < y1 ? y0 : y1) - (T)0.5 * (T)(ORDER + 1)) + 1, LO), LO + W - WN);
        T Sx0[WN], Sx1[WN], Sy0[WN], Sy1[WN];
#pragma unroll
        for (int w = 0; w < WN; w++) {
            const T px = (T)(gx + w), py = (T)(gy + w);
            Sx0[w] = bspline<ORDER>(x0 - px); Sx1[w] = bspline<ORDER>(x1 - px);
            Sy0[w] = bspline<ORDER>(y0 - py); Sy1[w] = bspline<ORDER>(y1 - py);
        }
        const T qp = q[p];
        const T c1 = c1s * qp, c2 = c2s * qp;
        const T c3 = v3 ? c3s * qp * v3[p] : (T)0;
        int col[WN];
        int64_t row[WN];
#pragma unroll
        for (int w = 0; w < WN; w++) { col[w] = wrapi(cx + gx + w, n1); row[w] = (int64_t)wrapi(cy + gy + w, n2) * n1; }
        auto add = [&](int c, int i, int j, T v) { atomicAdd(Jc[c] + row[j] + col[i], v); };
#pragma unroll
        for (int j = 0; j < WN; j++) {
            const T sy = (T)0.5 * (Sy0[j] + Sy1[j]);
            if (sy == (T)0) continue;
            T acc = (T)0;
#pragma unroll
            for (int i = 0; i < WN; i++) {
                acc += (Sx1[i] - Sx0[i]) * sy;
                if (acc != (T)0) add(0, i, j, c1 * acc);
            }
        }
#pragma unroll
        for (int i = 0; i < WN; i++) {
            const T sx = (T)0.5 * (Sx0[i] + Sx1[i]);
            if (sx == (T)0) continue;
            T acc = (T)0;
#pragma unroll
            for (int j = 0; j < WN; j++) {
                acc += (Sy1[j] - Sy0[j]) * sx;
                if (acc != (T)0) add(1, i, j, c2 * acc);
            }
        }
        if (c3 != (T)0) {
            // S1^0 S2^0/3 + S1^1 S2^0/6 + S1^0 S2^1/6 + S1^1 S2^1/3 = S1^0 a_j + S1^1 b_j
#pragma unroll
            for (int j = 0; j < WN; j++) {
                const T aj = (Sy0[j] + Sy0[j] + Sy1[j]) * ((T)1 / (T)6), bj = (Sy0[j] + Sy1[j] + Sy1[j]) * ((T)1 / (T)6);
#pragma unroll
                for (int i = 0; i < WN; i++) {
                    const T w3 = Sx0[i] * aj + Sx1[i] * bj;
                    if (w3 != (T)0) add(2, i, j, c3 * w3);
                }
            }
        }
    }
}

template <typename T, int ORDER>
__global__ void k_deposit3d(T* __restrict__ J1, T* __restrict__ J2, T* __restrict__ J3, int n1, int n2, int n3,
                            const int32_t* __restrict__ cell, const T* __restrict__ off0, const T* __restrict__ off1,
                            const T* __restrict__ q, int64_t np, T c1s, T c2s, T c3s, int* __restrict__ flag) {
    constexpr int W = Win<ORDER>::n, LO = Win<ORDER>::lo;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        T a0[3], a1[3];
        bool ok = true;
        const int ext[3] = {n1, n2, n3};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            c[a] = cell[3 * p + a];
            a0[a] = off0[3 * p + a];
            a1[a] = off1[3 * p + a];
            const T d = a1[a] - a0[a];
            ok = ok && a0[a] >= (T)0 && a0[a] < (T)1 && d > (T)-1 && d < (T)1 && c[a] >= 0 && c[a] < ext[a];
        }
        if (!ok) { atomicOr(flag, 1); continue; }
        T S0[3][W], dS[3][W];
        int idx[3][W];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int w = 0; w < W; w++) {
                const T gp = (T)(w + LO);
                S0[a][w] = bspline<ORDER>(a0[a] - gp);
                dS[a][w] = bspline<ORDER>(a1[a] - gp) - S0[a][w];
                idx[a][w] = wrapi(c[a] + LO + w, ext[a]);
            }
        const T qp = q[p];
        const T cc[3] = {c1s * qp, c2s * qp, c3s * qp};
        T* Jd[3] = {J1, J2, J3};
        // component a accumulates along axis a; (b, c) are the two transverse axes
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int b = (a + 1) % 3, e = (a + 2) % 3;
            for (int u = 0; u < W; u++)
                for (int v = 0; v < W; v++) {
                    const T tw = S0[b][u] * S0[e][v] + (T)0.5 * dS[b][u] * S0[e][v] + (T)0.5 * S0[b][u] * dS[e][v]
                               + dS[b][u] * dS[e][v] * ((T)1 / (T)3);
                    if (tw == (T)0) continue;
                    T acc = (T)0;
                    for (int i = 0; i < W; i++) {
                        acc += dS[a][i] * tw;
                        if (acc == (T)0) continue;
                        int ii[3];
                        ii[a] = idx[a][i]; ii[b] = idx[b][u]; ii[e] = idx[e][v];
                        atomicAdd(Jd[a] + ((int64_t)ii[2] * n2 + ii[1]) * n1 + ii[0], cc[a] * acc);
                    }
                }
        }
    }
}

template <typename T>
hyb_status deposit(hyb_grid* g, const int32_t* cell, const T* off_old, const T* off_new, const T* v3, const T* q,
                   int64_t np, int order) {
    const hyb_grid_desc& d = g->d;
    const size_t bytes = (size_t)g->cells * sizeof(T);
    for (int c = 0; c < 3; c++) HYB_CUDA_TRY(cudaMemsetAsync(g->J[c], 0, bytes, g->stream));
    if (np == 0) return HYB_OK;
    T* J1 = (T*)g->J[0]; T* J2 = (T*)g->J[1]; T* J3 = (T*)g->J[2];
    const int threads = kDepThreads;
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, g->device);
    int64_t want = (np + threads - 1) / threads;
    unsigned blocks = (unsigned)(want < (int64_t)dev_sms * 32 ? want : (int64_t)dev_sms * 32);
    if (blocks == 0) blocks = 1;
    if (d.dims == 2) {
        const T c1 = (T)(-1.0 / (d.dt * d.dx2)), c2 = (T)(-1.0 / (d.dt * d.dx1)), c3 = (T)(1.0 / (d.dx1 * d.dx2));
#define HYB_DEP2(O) k_deposit2d<T, O><<<blocks, threads, 0, g->stream>>>(J1, J2, J3, d.n1, d.n2, cell, off_old, off_new, v3, q, np, c1, c2, c3, g->dflag)
        if (order == 1) HYB_DEP2(1); else if (order == 2) HYB_DEP2(2); else HYB_DEP2(3);
#undef HYB_DEP2
    } else {
        const T c1 = (T)(-1.0 / (d.dt * d.dx2 * d.dx3)), c2 = (T)(-1.0 / (d.dt * d.dx1 * d.dx3)), c3 = (T)(-1.0 / (d.dt * d.dx1 * d.dx2));
#define HYB_DEP3(O) k_deposit3d<T, O><<<blocks, threads, 0, g->stream>>>(J1, J2, J3, d.n1, d.n2, d.n3, cell, off_old, off_new, q, np, c1, c2, c3, g->dflag)
        if (order == 1) HYB_DEP3(1); else if (order == 2) HYB_DEP3(2); else HYB_DEP3(3);
#undef HYB_DEP3
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

template hyb_status deposit<float>(hyb_grid*, const int32_t*, const float*, const float*, const float*, const float*, int64_t, int);
template hyb_status deposit<double>(hyb_grid*, const int32_t*, const double*, const double*, const double*, const double*, int64_t, int);

}  // namespace hyb
