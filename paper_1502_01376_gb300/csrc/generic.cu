// generic.cu -- three-pass hybrid advance for any precision, 2D or 3D:
//   (1) batched real FFT along x1 of E, B, j into a spectral scratch,
//   (2) per-k1-mode Faraday then Ampere updates with finite differences in
//       x2 (and x3) (Eqs. hybrid2db1-hybrid2de3; Sec. 2.4 for 3D),
//   (3) batched inverse real FFT of E, B back in place.
// For FP32 rows of 1024 points the Ampere update of (2) is folded into (3),
// which then reads the spectra of E, B, j and writes E, B (three launches).
// It also provides the row FFTs used by the standalone current processing and
// the diagnostics.  The x1 transform is a shared-memory Stockham FFT (radix 8,
// then one radix-4 or radix-2 pass; several short rows per block)
// of the n1/2-point complex sequence z[j] = x[2j] + i x[2j+1] followed by the
// standard even/odd split into the n1/2+1 real-input coefficients.
#include <algorithm>
#include <type_traits>

#include "hyb_internal.cuh"
#include "packed_dev.cuh"

namespace hyb {

constexpr int kRowThreads = 256;
constexpr int kModeRows = 8;          // per-mode kernels: blocks of 32 modes x 8 rows

struct RowPtrs { const void* p[9]; };
struct RowPtrsW { void* p[9]; };

// X[k] = 1/2 (Z[k] + Z*[M-k]) - i/2 W_N^k (Z[k] - Z*[M-k]),  k = 0..M.
// A block transforms RB = fft_rows_per_block(M) consecutive rows of one field.
template <typename Tin, typename T>
__global__ void __launch_bounds__(kRowThreads) k_rfft_rows(RowPtrs in, cplx<T>* __restrict__ out, int n1, int64_t rows,
                                                           const cplx<T>* __restrict__ twS, const cplx<T>* __restrict__ twN, int RB) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = n1 >> 1;
    C* src = reinterpret_cast<C*>(smem_raw);
    C* dst = src + fpad_size((size_t)RB * M);
    const int64_t row0 = (int64_t)blockIdx.x * RB;
    const int nrow = (int)((rows - row0) < RB ? (rows - row0) : RB);
    const int f = blockIdx.y;
    const Tin* x = reinterpret_cast<const Tin*>(in.p[f]) + row0 * n1;
    if constexpr (std::is_same<Tin, T>::value) {           // (x[2q], x[2q+1]) as one complex load
        const C* xc = reinterpret_cast<const C*>(x);
        for (int q = threadIdx.x; q < nrow * M; q += blockDim.x) src[fpad(q)] = xc[q];
    } else {
        for (int q = threadIdx.x; q < nrow * M; q += blockDim.x) src[fpad(q)] = mkc<C>((T)x[2 * q], (T)x[2 * q + 1]);
    }
    __syncthreads();
    stockham_rows<C, false>(src, dst, M, nrow, twS);
    C* X = out + ((int64_t)f * rows + row0) * (M + 1);
    const int lgH = 31 - __clz(M) - 1, H = M >> 1;
    // pairs (k, M - k) for k < M/2 of all rows (k = 0 gives X[0] and X[M]), then k = M/2 of each row:
    // X[k] = e - u, X[M-k] = conj(e + u), e = (Z[k] + Z*[M-k])/2, u = (i/2) W_N^k (Z[k] - Z*[M-k])
    for (int q = threadIdx.x; q < (nrow << lgH) + nrow; q += blockDim.x) {
        int r, k;
        if (q < (nrow << lgH)) { r = q >> lgH; k = q & (H - 1); } else { r = q - (nrow << lgH); k = H; }
        const C zk = src[fpad(r * M + k)];
        const C zmc = cconj(src[fpad(r * M + ((M - k) & (M - 1)))]);
        const C e = cscale(cadd(zk, zmc), (T)0.5);
        const C wd = cmul(twN[k], csub(zk, zmc));
        C* Xr = X + (size_t)r * (M + 1);
        Xr[k] = mkc<C>(e.x + (T)0.5 * wd.y, e.y - (T)0.5 * wd.x);
        if (k != H) Xr[M - k] = mkc<C>(e.x - (T)0.5 * wd.y, -(e.y + (T)0.5 * wd.x));
    }
}

// inverse of the above: Z[k] = E + i O, E = (X[k] + X*[M-k])/2, O = conj(W_N^k)(X[k] - X*[M-k])/2,
// z = IDFT_M(Z) / M, x[2j] = Re z[j], x[2j+1] = Im z[j].  DC/Nyquist imaginary parts are dropped.
template <typename T, typename Tout>
__global__ void __launch_bounds__(kRowThreads) k_irfft_rows(const cplx<T>* __restrict__ in, RowPtrsW out, int n1, int64_t rows,
                                                            const cplx<T>* __restrict__ twS, const cplx<T>* __restrict__ twN,
                                                            int in_field0, int RB) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = n1 >> 1;
    C* src = reinterpret_cast<C*>(smem_raw);
    C* dst = src + fpad_size((size_t)RB * M);
    const int64_t row0 = (int64_t)blockIdx.x * RB;
    const int nrow = (int)((rows - row0) < RB ? (rows - row0) : RB);
    const int f = blockIdx.y;
    const C* X = in + ((int64_t)(in_field0 + f) * rows + row0) * (M + 1);
    const int lgH = 31 - __clz(M) - 1, H = M >> 1;
    // pairs (k, M - k) for k < M/2 (k = 0 reads X[0] and X[M]), then k = M/2 of each row:
    // Z[k] = E + iO, Z[M-k] = conj(E - iO)
    for (int q = threadIdx.x; q < (nrow << lgH) + nrow; q += blockDim.x) {
        int r, k;
        if (q < (nrow << lgH)) { r = q >> lgH; k = q & (H - 1); } else { r = q - (nrow << lgH); k = H; }
        const C* Xr = X + (size_t)r * (M + 1);
        C xk = Xr[k], xm = Xr[M - k];
        if (k == 0) { xk.y = 0; xm.y = 0; }
        const C xmc = cconj(xm);
        const C e = cscale(cadd(xk, xmc), (T)0.5);
        const C o = cscale(cmulc(csub(xk, xmc), twN[k]), (T)0.5);
        src[fpad(r * M + k)] = mkc<C>(e.x - o.y, e.y + o.x);
        if (k != 0 && k != H) src[fpad(r * M + M - k)] = mkc<C>(e.x + o.y, o.x - e.y);
    }
    __syncthreads();
    stockham_rows<C, true>(src, dst, M, nrow, twS);
    Tout* x = reinterpret_cast<Tout*>(out.p[f]) + row0 * n1;
    const T inv = (T)1 / (T)M;
    if constexpr (std::is_same<Tout, T>::value) {
        C* xc = reinterpret_cast<C*>(x);
        for (int q = threadIdx.x; q < nrow * M; q += blockDim.x) xc[q] = cscale(src[fpad(q)], inv);
    } else {
        for (int q = threadIdx.x; q < nrow * M; q += blockDim.x) {
            const C z = src[fpad(q)];
            x[2 * q] = (Tout)(z.x * inv);
            x[2 * q + 1] = (Tout)(z.y * inv);
        }
    }
}

// ---------------------------------------------------------------- n1 = 1024, FP32: register-resident row FFT
// The 512-point complex FFT of z[j] = x[2j] + i x[2j+1], factored 8 x 8 x 8 over 64 threads per
// row (8 points each), the exchanges through shared memory, then the real-input split in
// (k, M - k) pairs:
//   S1  thread t: z[t + 64 n], DFT8 over n -> k1, twiddle W_512^{t k1}          -> A(k1, t)
//   S2  (t0, k1) = (t & 7, t >> 3): A(k1, t0 + 8 t1), DFT8 over t1 -> k2,
//       twiddle W_64^{t0 k2}                                                  -> B[9 (8 k1 + k2) + t0]
//   S3  (k1, k2) = (t >> 3, t & 7): B[9 (8 k1 + k2) + t0], DFT8 over t0 -> Z[k1 + 8 k2 + 64 k3]
// A(k, t) is stored at 72 k + t and Z[k] at a swizzled position (both against bank conflicts); the
// twiddles of S1 and S2 come from a table laid out in the order the threads read them.
// The inverse runs the stages
// transposed with conjugate twiddles.  Four rows per block, one named barrier per row.
constexpr int kRows1k = 4;
constexpr int kBuf1k = 576;
// Z[k] at k with bits 2 and 1 flipped by bits 4 and 5: a half-warp's 8-byte accesses of the S3
// scatter (lanes over bits 0, 3, 4, 5 of k) and of the split (16 consecutive k) both reach 16
// different bank pairs
__device__ __forceinline__ int zp1k(int k) { return k ^ (((k >> 4) & 1) << 2) ^ (((k >> 5) & 1) << 1); }
// stage-1 output (k1, t) position
__device__ __forceinline__ int ap1k(int k, int t) { return 72 * k + t; }
__device__ __forceinline__ float2 cm(float2 a, float2 b) { return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)); }
__device__ __forceinline__ float2 cmc(float2 a, float2 b) { return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y)); }

// Persistent: each 64-thread team (four per block) walks the rows j = team, team + teams, ... of all
// fields (field j / rows), holding the next row's samples in registers while it transforms the
// current one, so that every team keeps a row of loads in flight.
__global__ void __launch_bounds__(256, 3) k_rfft1024(RowPtrs in, float2* __restrict__ out, int64_t rows, int nf,
                                                  const float2* __restrict__ tw8, const float2* __restrict__ twN) {
    __shared__ float2 sbuf[kRows1k][2][kBuf1k];
    const int L = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int64_t total = rows * nf, teams = (int64_t)gridDim.x * kRows1k;
    float2* A = sbuf[L][0];
    float2* B = sbuf[L][1];
    auto lsync = [&]() { asm volatile("bar.sync %0, %1;" :: "r"(1 + L), "r"(64) : "memory"); };
    float2 nx[8], w1[8], w2[8];
#pragma unroll
    for (int k = 1; k < 8; k++) {
        w1[k] = tw8[(k - 1) * 64 + t];
        w2[k] = tw8[448 + (k - 1) * 8 + (t & 7)];
    }
    auto fetch = [&](int64_t j) {
        const int f = (int)(j / rows);
        const float2* z = reinterpret_cast<const float2*>(in.p[f]) + (j - (int64_t)f * rows) * 512;
#pragma unroll
        for (int n = 0; n < 8; n++) nx[n] = __ldcs(z + t + 64 * n);
    };
    int64_t j = (int64_t)blockIdx.x * kRows1k + L;
    if (j < total) fetch(j);
    for (; j < total; j += teams) {
        float2 v[8];
#pragma unroll
        for (int n = 0; n < 8; n++) v[n] = nx[n];
        if (j + teams < total) fetch(j + teams);
        dft8x<false>(v);
#pragma unroll
        for (int k = 1; k < 8; k++) v[k] = cm(v[k], w1[k]);
        lsync();                     // the previous row's split has read A
#pragma unroll
        for (int k = 0; k < 8; k++) A[ap1k(k, t)] = v[k];
        lsync();
        {
            const int t0 = t & 7, k1 = t >> 3;
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = A[ap1k(k1, t0 + 8 * n)];
            dft8x<false>(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = cm(v[k], w2[k]);
#pragma unroll
            for (int k = 0; k < 8; k++) B[9 * (8 * k1 + k) + t0] = v[k];
        }
        lsync();
        {
            const int k1 = t >> 3, k2 = t & 7;
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = B[9 * (8 * k1 + k2) + n];
            dft8x<false>(v);
#pragma unroll
            for (int k = 0; k < 8; k++) A[zp1k(k1 + 8 * k2 + 64 * k)] = v[k];
        }
        lsync();
        float2* X = out + j * 513;   // [field][row][513], j = field * rows + row
        // X[k] = e - u, X[M-k] = conj(e + u), e = (Z[k] + Z*[M-k])/2, u = (i/2) W_N^k (Z[k] - Z*[M-k])
        auto pair = [&](int k) {
            const float2 zk = A[zp1k(k)], zm = A[zp1k((512 - k) & 511)];
            const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 wd = cm(twN[k], make_float2(zk.x - zm.x, zk.y + zm.y));
            X[k] = make_float2(e.x + 0.5f * wd.y, e.y - 0.5f * wd.x);
            if (k != 256) X[512 - k] = make_float2(e.x - 0.5f * wd.y, -(e.y + 0.5f * wd.x));
        };
#pragma unroll
        for (int m = 0; m < 4; m++) pair(t + 64 * m);
        if (t == 0) pair(256);
    }
}

// Inverse of one row from its spectrum, X[k] = ld(k) for k = 0..M (the stages of k_rfft1024 in
// reverse with conjugate twiddles); z_out receives the 1024 real samples (nullptr: dead row).
template <class Ld>
__device__ __forceinline__ void irfft1024_row(float2* A, float2* B, int L, int t, float2* __restrict__ z_out,
                                              const float2* __restrict__ tw8, const float2* __restrict__ twN, Ld ld) {
    auto lsync = [&]() { asm volatile("bar.sync %0, %1;" :: "r"(1 + L), "r"(64) : "memory"); };
    {
        // Z[k] = E + iO, Z[M-k] = conj(E - iO), E = (X[k] + X*[M-k])/2, O = conj(W_N^k)(X[k] - X*[M-k])/2;
        // the imaginary parts of X[0] and X[M] are dropped
        auto pair = [&](int k) {
            float2 xk = ld(k);
            float2 xm = k == 256 ? xk : ld(512 - k);        // each mode loaded once
            if (k == 0) { xk.y = 0.f; xm.y = 0.f; }
            const float2 e = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y - xm.y));
            const float2 o = cmc(make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y + xm.y)), twN[k]);
            A[zp1k(k)] = make_float2(e.x - o.y, e.y + o.x);
            if (k != 0 && k != 256) A[zp1k(512 - k)] = make_float2(e.x + o.y, o.x - e.y);
        };
#pragma unroll
        for (int m = 0; m < 4; m++) pair(t + 64 * m);
        if (t == 0) pair(256);
    }
    lsync();
    float2 v[8];
    {
        const int k1 = t >> 3, k2 = t & 7;
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = A[zp1k(k1 + 8 * k2 + 64 * k)];
        dft8x<true>(v);
#pragma unroll
        for (int n = 0; n < 8; n++) B[9 * (8 * k1 + k2) + n] = v[n];
    }
    lsync();
    {
        const int t0 = t & 7, k1 = t >> 3;
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = B[9 * (8 * k1 + k) + t0];
#pragma unroll
        for (int k = 1; k < 8; k++) v[k] = cmc(v[k], tw8[448 + (k - 1) * 8 + t0]);
        dft8x<true>(v);
#pragma unroll
        for (int n = 0; n < 8; n++) A[ap1k(k1, t0 + 8 * n)] = v[n];
    }
    lsync();
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = A[ap1k(k, t)];
#pragma unroll
    for (int k = 1; k < 8; k++) v[k] = cmc(v[k], tw8[(k - 1) * 64 + t]);
    dft8x<true>(v);
    if (z_out) {
        const float inv = 1.f / 512.f;
#pragma unroll
        for (int n = 0; n < 8; n++) z_out[t + 64 * n] = make_float2(v[n].x * inv, v[n].y * inv);
    }
}

__global__ void __launch_bounds__(256) k_irfft1024(const float2* __restrict__ in, RowPtrsW out, int64_t rows,
                                                   const float2* __restrict__ tw8, const float2* __restrict__ twN,
                                                   int in_field0) {
    __shared__ float2 sbuf[kRows1k][2][kBuf1k];
    const int L = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int64_t row = (int64_t)blockIdx.x * kRows1k + L;
    const bool live = row < rows;
    const int f = blockIdx.y;
    const float2* X = in + ((int64_t)(in_field0 + f) * rows + (live ? row : 0)) * 513;
    float2* z = live ? reinterpret_cast<float2*>(out.p[f]) + row * 512 : nullptr;
    irfft1024_row(sbuf[L][0], sbuf[L][1], L, t, z, tw8, twN, [&](int k) { return X[k]; });
}

// Ampere (Eqs. hybrid2de1-hybrid2de3; the x3 differences of Sec. 2.4) fused into the inverse
// transform of E, B: blocks of kRows1k rows of one field, the six fields of a row group in
// consecutive blocks so that the B rows three of them read come from L2.  Fields 0-2 apply Ampere
// to E_f mode by mode as they load it (Sm = -conj(S) = c dt sigma-):
//   E1 += a2 d2-B3 - a3 d3-B2 - cj1 J1;  E2 += a3 d3-B1 - Sm B3 - cj J2;  E3 += Sm B2 - a2 d2-B1 - cj J3
// fields 3-5 invert B.  Without WB the spectral scratch is only read; with WB (k1-resident
// state) the updated E spectrum is also stored back in place (each mode of a row is loaded once,
// by the block of that row and field).
template <bool D3, bool WB>
__global__ void __launch_bounds__(256, 3) k_ampere_irfft1024(float2* __restrict__ spec, RowPtrsW out, int64_t rows, int n2, int n3,
                                                          const float2* __restrict__ tw8, const float2* __restrict__ twN,
                                                          const float2* __restrict__ S, const float* __restrict__ cj1,
                                                          const float* __restrict__ cj, float a2, float a3) {
    __shared__ float2 sbuf[kRows1k][2][kBuf1k];
    const int L = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int f = blockIdx.x % 6;
    const int64_t row = (int64_t)(blockIdx.x / 6) * kRows1k + L;
    const bool live = row < rows;
    const int64_t r = live ? row : 0;
    const int64_t i3 = r / n2;
    const int i2 = (int)(r - i3 * n2);
    const int64_t fs = rows * 513;
    float2* Xr = spec + r * 513;                                                  // field 0 of row r
    const float2* Xm2 = spec + (i3 * n2 + (i2 == 0 ? n2 - 1 : i2 - 1)) * 513;     // row i2 - 1
    const float2* Xm3 = spec + ((D3 ? (i3 == 0 ? n3 - 1 : i3 - 1) : i3) * n2 + i2) * 513;   // row i3 - 1
    float2* z = live ? reinterpret_cast<float2*>(out.p[f]) + row * 512 : nullptr;
    auto sub = [](float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); };
    auto axpy = [](float2 y, float s, float2 x) { return make_float2(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y)); };
    auto keep = [&](float2* at, float2 e) {
        if (WB && live) *at = e;
        return e;
    };
    if (f == 0) {
        irfft1024_row(sbuf[L][0], sbuf[L][1], L, t, z, tw8, twN, [&](int k) {
            float2 e = axpy(Xr[k], a2, sub(Xr[5 * fs + k], Xm2[5 * fs + k]));
            if (D3) e = axpy(e, -a3, sub(Xr[4 * fs + k], Xm3[4 * fs + k]));
            return keep(Xr + k, axpy(e, -cj1[k], Xr[6 * fs + k]));
        });
    } else if (f == 1) {
        irfft1024_row(sbuf[L][0], sbuf[L][1], L, t, z, tw8, twN, [&](int k) {
            const float2 s = S[k], b3 = Xr[5 * fs + k];
            // - Sm B3 = conj(S) B3
            float2 e = Xr[fs + k];
            e = make_float2(e.x + (s.x * b3.x + s.y * b3.y), e.y + (s.x * b3.y - s.y * b3.x));
            if (D3) e = axpy(e, a3, sub(Xr[3 * fs + k], Xm3[3 * fs + k]));
            return keep(Xr + fs + k, axpy(e, -cj[k], Xr[7 * fs + k]));
        });
    } else if (f == 2) {
        irfft1024_row(sbuf[L][0], sbuf[L][1], L, t, z, tw8, twN, [&](int k) {
            const float2 s = S[k], b2 = Xr[4 * fs + k];
            // + Sm B2 = - conj(S) B2
            float2 e = Xr[2 * fs + k];
            e = make_float2(e.x - (s.x * b2.x + s.y * b2.y), e.y - (s.x * b2.y - s.y * b2.x));
            e = axpy(e, -a2, sub(Xr[3 * fs + k], Xm2[3 * fs + k]));
            return keep(Xr + 2 * fs + k, axpy(e, -cj[k], Xr[8 * fs + k]));
        });
    } else {
        const float2* X = Xr + f * fs;
        irfft1024_row(sbuf[L][0], sbuf[L][1], L, t, z, tw8, twN, [&](int k) { return X[k]; });
    }
}

template <typename T>
static size_t row_fft_smem(int n1, int RB) { return sizeof(cplx<T>) * 2 * fpad_size((size_t)RB * (n1 / 2)); }
template <typename T>
static size_t max_row_fft_smem() {
    size_t m = 0;
    for (int n1 = 8; n1 <= 8192; n1 *= 2) m = std::max(m, row_fft_smem<T>(n1, fft_rows_per_block(n1 / 2)));
    return m;
}

template <typename Tin, typename T>
static cudaError_t launch_rfft(const RowPtrs& p, int nf, cplx<T>* out, int n1, int64_t rows, const ModeTables<T>& t, cudaStream_t s) {
    if constexpr (std::is_same<Tin, float>::value && std::is_same<T, float>::value) {
        if (n1 == 1024) {
            const cudaError_t carve = func_attr_once((const void*)k_rfft1024, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (carve != cudaSuccess) return carve;
            const int resident = resident_grid((const void*)k_rfft1024, 256, 0);
            const int64_t blocks = std::min<int64_t>((rows * nf + kRows1k - 1) / kRows1k, resident);
            k_rfft1024<<<(unsigned)blocks, 256, 0, s>>>(p, out, rows, nf, t.tw8, t.twN);
            return cudaGetLastError();
        }
    }
    const int RB = fft_rows_per_launch(n1 / 2, rows * nf);
    const size_t smem = row_fft_smem<T>(n1, RB);
    auto kern = k_rfft_rows<Tin, T>;
    // once per kernel and device: room for the largest row block any n1 up to 8192 asks for
    const cudaError_t attr = func_attr_once((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_row_fft_smem<T>());
    if (attr != cudaSuccess) return attr;
    dim3 grid((unsigned)((rows + RB - 1) / RB), nf);
    kern<<<grid, kRowThreads, smem, s>>>(p, out, n1, rows, t.twS, t.twN, RB);
    return cudaGetLastError();
}

template <typename T, typename Tout>
static cudaError_t launch_irfft(const cplx<T>* in, int f0, const RowPtrsW& p, int nf, int n1, int64_t rows, const ModeTables<T>& t, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value && std::is_same<Tout, float>::value) {
        if (n1 == 1024) {
            const cudaError_t carve = func_attr_once((const void*)k_irfft1024, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (carve != cudaSuccess) return carve;
            k_irfft1024<<<dim3((unsigned)((rows + kRows1k - 1) / kRows1k), nf), 256, 0, s>>>(in, p, rows, t.tw8, t.twN, f0);
            return cudaGetLastError();
        }
    }
    const int RB = fft_rows_per_launch(n1 / 2, rows * nf);
    const size_t smem = row_fft_smem<T>(n1, RB);
    auto kern = k_irfft_rows<T, Tout>;
    // once per kernel and device: room for the largest row block any n1 up to 8192 asks for
    const cudaError_t attr = func_attr_once((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_row_fft_smem<T>());
    if (attr != cudaSuccess) return attr;
    dim3 grid((unsigned)((rows + RB - 1) / RB), nf);
    kern<<<grid, kRowThreads, smem, s>>>(in, p, n1, rows, t.twS, t.twN, f0, RB);
    return cudaGetLastError();
}

template <typename Tin, typename T>
cudaError_t rfft_rows(const Tin* in, cplx<T>* out, int n1, int64_t rows, const ModeTables<T>& t, cudaStream_t s) {
    RowPtrs p{};
    p.p[0] = in;
    return launch_rfft<Tin, T>(p, 1, out, n1, rows, t, s);
}

template <typename T, typename Tout>
cudaError_t irfft_rows(const cplx<T>* in, Tout* out, int n1, int64_t rows, const ModeTables<T>& t, cudaStream_t s) {
    RowPtrsW p{};
    p.p[0] = out;
    return launch_irfft<T, Tout>(in, 0, p, 1, n1, rows, t, s);
}

template cudaError_t rfft_rows<float, float>(const float*, float2*, int, int64_t, const ModeTables<float>&, cudaStream_t);
template cudaError_t rfft_rows<double, double>(const double*, double2*, int, int64_t, const ModeTables<double>&, cudaStream_t);
template cudaError_t rfft_rows<float, double>(const float*, double2*, int, int64_t, const ModeTables<double>&, cudaStream_t);
template cudaError_t irfft_rows<float, float>(const float2*, float*, int, int64_t, const ModeTables<float>&, cudaStream_t);
template cudaError_t irfft_rows<double, double>(const double2*, double*, int, int64_t, const ModeTables<double>&, cudaStream_t);

// ----------------------------------------------------------------------------
// per-mode updates; spec layout [9][rows][nk], fields E1 E2 E3 B1 B2 B3 J1 J2 J3,
// row = i3 * n2 + i2.
// Faraday:  B1 -= a2 d2+E3 - a3 d3+E2;  B2 -= a3 d3+E1 - S E3;  B3 -= S E2 - a2 d2+E1
template <typename T, bool D3>
__global__ void __launch_bounds__(kRowThreads) k_faraday(cplx<T>* __restrict__ spec, int nk, int n2, int n3, int64_t rows,
                                                         const cplx<T>* __restrict__ S, T a2, T a3) {
    using C = cplx<T>;
    // block (32 modes) x (8 rows of one x3 plane); consecutive blocks walk the modes of a
    // row group first: blockIdx.x = (i3 * g2 + i2 / 8) * nch + k / 32
    const int g2 = (n2 + kModeRows - 1) / kModeRows, nch = (nk + 31) / 32;
    const int rg = blockIdx.x / nch, ch = blockIdx.x - rg * nch;
    const int i3 = rg / g2, i2 = (rg - i3 * g2) * kModeRows + threadIdx.y;
    const int k = ch * 32 + threadIdx.x;
    if (i2 >= n2 || k >= nk) return;
    const int64_t r = (int64_t)i3 * n2 + i2;
    const int64_t rp2 = (int64_t)i3 * n2 + (i2 + 1 == n2 ? 0 : i2 + 1);
    const int64_t rp3 = D3 ? (int64_t)(i3 + 1 == n3 ? 0 : i3 + 1) * n2 + i2 : r;
    const int64_t fs = rows * nk;
    C* E1 = spec; C* E2 = spec + fs; C* E3 = spec + 2 * fs;
    C* B1 = spec + 3 * fs; C* B2 = spec + 4 * fs; C* B3 = spec + 5 * fs;
    {
        const int64_t i = r * nk + k, ip2 = rp2 * nk + k, ip3 = rp3 * nk + k;
        C e1 = E1[i], e2 = E2[i], e3 = E3[i], s = S[k];
        C d2e3 = cscale(csub(E3[ip2], e3), a2);
        C d2e1 = cscale(csub(E1[ip2], e1), a2);
        C b1 = B1[i], b2 = B2[i], b3 = B3[i];
        b1 = csub(b1, d2e3);
        b2 = cadd(b2, cmul(s, e3));
        b3 = csub(b3, csub(cmul(s, e2), d2e1));
        if (D3) {
            C d3e2 = cscale(csub(E2[ip3], e2), a3);
            C d3e1 = cscale(csub(E1[ip3], e1), a3);
            b1 = cadd(b1, d3e2);
            b2 = csub(b2, d3e1);
        }
        B1[i] = b1; B2[i] = b2; B3[i] = b3;
    }
}

// B^n = B^{n-1/2} + (1/2) Faraday(E^n) per mode, from the resident spectra into out (3 spectral
// fields): the time-centred B a particle push gathers, without advancing the state
template <typename T, bool D3>
__global__ void __launch_bounds__(kRowThreads) k_faraday_half(const cplx<T>* __restrict__ spec, cplx<T>* __restrict__ out, int nk,
                                                              int n2, int n3, int64_t rows, const cplx<T>* __restrict__ S, T a2, T a3) {
    using C = cplx<T>;
    const int g2 = (n2 + kModeRows - 1) / kModeRows, nch = (nk + 31) / 32;
    const int rg = blockIdx.x / nch, ch = blockIdx.x - rg * nch;
    const int i3 = rg / g2, i2 = (rg - i3 * g2) * kModeRows + threadIdx.y;
    const int k = ch * 32 + threadIdx.x;
    if (i2 >= n2 || k >= nk) return;
    const int64_t r = (int64_t)i3 * n2 + i2;
    const int64_t rp2 = (int64_t)i3 * n2 + (i2 + 1 == n2 ? 0 : i2 + 1);
    const int64_t rp3 = D3 ? (int64_t)(i3 + 1 == n3 ? 0 : i3 + 1) * n2 + i2 : r;
    const int64_t fs = rows * nk;
    const C* E1 = spec; const C* E2 = spec + fs; const C* E3 = spec + 2 * fs;
    const C* B1 = spec + 3 * fs; const C* B2 = spec + 4 * fs; const C* B3 = spec + 5 * fs;
    const int64_t i = r * nk + k, ip2 = rp2 * nk + k, ip3 = rp3 * nk + k;
    const C e1 = E1[i], e2 = E2[i], e3 = E3[i], s = S[k];
    const T h = (T)0.5;
    // the increments of k_faraday, halved
    C d1 = cscale(csub(E3[ip2], e3), -a2);
    C d2 = cmul(s, e3);
    C d3 = csub(cscale(csub(E1[ip2], e1), a2), cmul(s, e2));
    if (D3) {
        d1 = cadd(d1, cscale(csub(E2[ip3], e2), a3));
        d2 = csub(d2, cscale(csub(E1[ip3], e1), a3));
    }
    out[i] = cadd(B1[i], cscale(d1, h));
    out[fs + i] = cadd(B2[i], cscale(d2, h));
    out[2 * fs + i] = cadd(B3[i], cscale(d3, h));
}

// Ampere (Sm = c dt sigma- = -conj(S)):
//   E1 += a2 d2-B3 - a3 d3-B2 - cj1 J1;  E2 += a3 d3-B1 - Sm B3 - cj J2;  E3 += Sm B2 - a2 d2-B1 - cj J3
template <typename T, bool D3>
__global__ void __launch_bounds__(kRowThreads) k_ampere(cplx<T>* __restrict__ spec, int nk, int n2, int n3, int64_t rows,
                                                        const cplx<T>* __restrict__ S, const T* __restrict__ cj1,
                                                        const T* __restrict__ cj, T a2, T a3) {
    using C = cplx<T>;
    const int g2 = (n2 + kModeRows - 1) / kModeRows, nch = (nk + 31) / 32;
    const int rg = blockIdx.x / nch, ch = blockIdx.x - rg * nch;
    const int i3 = rg / g2, i2 = (rg - i3 * g2) * kModeRows + threadIdx.y;
    const int k = ch * 32 + threadIdx.x;
    if (i2 >= n2 || k >= nk) return;
    const int64_t r = (int64_t)i3 * n2 + i2;
    const int64_t rm2 = (int64_t)i3 * n2 + (i2 == 0 ? n2 - 1 : i2 - 1);
    const int64_t rm3 = D3 ? (int64_t)(i3 == 0 ? n3 - 1 : i3 - 1) * n2 + i2 : r;
    const int64_t fs = rows * nk;
    C* E1 = spec; C* E2 = spec + fs; C* E3 = spec + 2 * fs;
    const C* B1 = spec + 3 * fs; const C* B2 = spec + 4 * fs; const C* B3 = spec + 5 * fs;
    const C* J1 = spec + 6 * fs; const C* J2 = spec + 7 * fs; const C* J3 = spec + 8 * fs;
    {
        const int64_t i = r * nk + k, im2 = rm2 * nk + k, im3 = rm3 * nk + k;
        C s = S[k];
        C sm = mkc<C>(-s.x, s.y);          // -conj(S)
        C b1 = B1[i], b2 = B2[i], b3 = B3[i];
        C d2b3 = cscale(csub(b3, B3[im2]), a2);
        C d2b1 = cscale(csub(b1, B1[im2]), a2);
        C e1 = cadd(E1[i], d2b3);
        C e2 = csub(E2[i], cmul(sm, b3));
        C e3 = csub(cadd(E3[i], cmul(sm, b2)), d2b1);
        if (D3) {
            C d3b2 = cscale(csub(b2, B2[im3]), a3);
            C d3b1 = cscale(csub(b1, B1[im3]), a3);
            e1 = csub(e1, d3b2);
            e2 = cadd(e2, d3b1);
        }
        const T c1 = cj1[k], c = cj[k];
        E1[i] = csub(e1, cscale(J1[i], c1));
        E2[i] = csub(e2, cscale(J2[i], c));
        E3[i] = csub(e3, cscale(J3[i], c));
    }
}

template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_scale_rows(cplx<T>* __restrict__ spec, int nk, int64_t rows, const T* __restrict__ fac) {
    const int64_t r = blockIdx.x;
    cplx<T>* X = spec + ((int64_t)blockIdx.y * rows + r) * nk;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) X[k] = cscale(X[k], fac[k]);
}

template <typename T> static const ModeTables<T>& tables(hyb_grid* g);
template <> const ModeTables<float>& tables<float>(hyb_grid* g) { return g->tf; }
template <> const ModeTables<double>& tables<double>(hyb_grid* g) { return g->td; }

// FP32 n1 = 1024 off the DFT-GEMM path: Ampere runs inside the inverse transform
static bool amp_fused(const hyb_grid* g) { return g->d.precision == 32 && g->d.n1 == 1024 && g->path < 3 && g->d.dims != 20; }

template <typename T>
hyb_status generic_advance(hyb_grid* g, int nsteps) {
    using C = cplx<T>;
    const ModeTables<T>& t = tables<T>(g);
    const int n1 = g->d.n1, nk = g->nk;
    const int64_t rows = g->rows;
    C* spec = reinterpret_cast<C*>(g->spec);
    const void* src9[9];
    for (int c = 0; c < 3; c++) { src9[c] = g->E[c]; src9[3 + c] = g->B[c]; src9[6 + c] = g->J[c]; }
    RowPtrsW fout{};
    for (int c = 0; c < 3; c++) { fout.p[c] = g->E[c]; fout.p[3 + c] = g->B[c]; }
    const T a2 = (T)(g->d.dt / g->d.dx2);
    const T a3 = (T)(g->d.dims == 3 ? g->d.dt / g->d.dx3 : 0.0);
    const bool d3 = g->d.dims == 3;
    for (int s = 0; s < nsteps; s++) {
        if (g->ev_start) HYB_CUDA_TRY(cudaEventRecord(g->ev_start, g->stream));
        // k1-resident state: the spectra of E and B left by the previous step are this step's
        // input, so only j is transformed (the first step after hyb_set_resident imports E, B)
        const int f0 = (g->resident && !g->res_stale) ? 6 : 0;
        RowPtrs fin{};
        for (int c = f0; c < 9; c++) fin.p[c - f0] = src9[c];
        C* spec_in = spec + (int64_t)f0 * rows * nk;
        if (g->path >= 3) {
            const float* fsrc[9];
            for (int c = f0; c < 9; c++) fsrc[c - f0] = (const float*)src9[c];
            hyb_status st = dftgemm_forward(g, fsrc, 9 - f0, reinterpret_cast<float2*>(spec_in));
            if (st != HYB_OK) return st;
        } else {
            HYB_CUDA_TRY((launch_rfft<T, T>(fin, 9 - f0, spec_in, n1, rows, t, g->stream)));
        }
        if (g->resident) g->res_stale = false;
        const dim3 mgrid((unsigned)((int64_t)g->d.n3 * ((g->d.n2 + kModeRows - 1) / kModeRows) * ((nk + 31) / 32))), mblk(32, kModeRows);
        if constexpr (std::is_same<T, float>::value) {
            if (amp_fused(g)) {
                float2* sp = reinterpret_cast<float2*>(spec);
                const unsigned nb = (unsigned)((rows + kRows1k - 1) / kRows1k) * 6u;
                const int n3 = d3 ? g->d.n3 : 1;
                if (d3) k_faraday<T, true><<<mgrid, mblk, 0, g->stream>>>(spec, nk, g->d.n2, n3, rows, t.S, a2, a3);
                else k_faraday<T, false><<<mgrid, mblk, 0, g->stream>>>(spec, nk, g->d.n2, 1, rows, t.S, a2, a3);
                auto amp = d3 ? (g->resident ? k_ampere_irfft1024<true, true> : k_ampere_irfft1024<true, false>)
                              : (g->resident ? k_ampere_irfft1024<false, true> : k_ampere_irfft1024<false, false>);
                amp<<<nb, 256, 0, g->stream>>>(sp, fout, rows, g->d.n2, n3, t.tw8, t.twN, t.S, t.cj1, t.cj, a2, a3);
                HYB_CUDA_TRY(cudaGetLastError());
                if (g->ev_stop) HYB_CUDA_TRY(cudaEventRecord(g->ev_stop, g->stream));
                continue;
            }
        }
        if (d3) {
            k_faraday<T, true><<<mgrid, mblk, 0, g->stream>>>(spec, nk, g->d.n2, g->d.n3, rows, t.S, a2, a3);
            k_ampere<T, true><<<mgrid, mblk, 0, g->stream>>>(spec, nk, g->d.n2, g->d.n3, rows, t.S, t.cj1, t.cj, a2, a3);
        } else {
            k_faraday<T, false><<<mgrid, mblk, 0, g->stream>>>(spec, nk, g->d.n2, 1, rows, t.S, a2, a3);
            k_ampere<T, false><<<mgrid, mblk, 0, g->stream>>>(spec, nk, g->d.n2, 1, rows, t.S, t.cj1, t.cj, a2, a3);
        }
        HYB_CUDA_TRY(cudaGetLastError());
        if (g->path >= 3) {
            float* f6[6];
            for (int c = 0; c < 6; c++) f6[c] = (float*)fout.p[c];
            hyb_status st = dftgemm_inverse(g, reinterpret_cast<const float2*>(spec), 6, f6);
            if (st != HYB_OK) return st;
        } else {
            HYB_CUDA_TRY((launch_irfft<T, T>(spec, 0, fout, 6, n1, rows, t, g->stream)));
        }
        if (g->ev_stop) HYB_CUDA_TRY(cudaEventRecord(g->ev_stop, g->stream));
    }
    return HYB_OK;
}

template <typename T>
hyb_status generic_process_current(hyb_grid* g, bool corr, bool filt) {
    using C = cplx<T>;
    const ModeTables<T>& t = tables<T>(g);
    const int n1 = g->d.n1, nk = g->nk;
    const int64_t rows = g->rows;
    // the j part of the scratch (its last three fields), so that a k1-resident E, B survives
    C* spec = reinterpret_cast<C*>(g->spec) + (int64_t)(g->spec_fields - 3) * rows * nk;
    int nf = filt ? 3 : 1;
    RowPtrs fin{};
    RowPtrsW fout{};
    for (int c = 0; c < nf; c++) { fin.p[c] = g->J[c]; fout.p[c] = g->J[c]; }
    HYB_CUDA_TRY((launch_rfft<T, T>(fin, nf, spec, n1, rows, t, g->stream)));
    if (filt) {
        dim3 grid((unsigned)rows, 3);
        k_scale_rows<T><<<grid, kRowThreads, 0, g->stream>>>(spec, nk, rows, t.filt);
    }
    if (corr) {
        dim3 grid((unsigned)rows, 1);
        k_scale_rows<T><<<grid, kRowThreads, 0, g->stream>>>(spec, nk, rows, t.corr);
    }
    HYB_CUDA_TRY(cudaGetLastError());
    HYB_CUDA_TRY((launch_irfft<T, T>(spec, 0, fout, nf, n1, rows, t, g->stream)));
    return HYB_OK;
}

// k1-resident state: transform the bound E, B into their spectra (the import a resident step
// does when its state is stale)
template <typename T>
hyb_status generic_resident_import(hyb_grid* g) {
    using C = cplx<T>;
    const ModeTables<T>& t = tables<T>(g);
    RowPtrs fin{};
    for (int c = 0; c < 3; c++) { fin.p[c] = g->E[c]; fin.p[3 + c] = g->B[c]; }
    HYB_CUDA_TRY((launch_rfft<T, T>(fin, 6, reinterpret_cast<C*>(g->spec), g->d.n1, g->rows, t, g->stream)));
    g->res_stale = false;
    return HYB_OK;
}

// B^n = B^{n-1/2} + (1/2) Faraday(E^n) from the resident spectra, into the real arrays Bh (the
// spectral j slots serve as scratch: the next step transforms j again)
template <typename T>
hyb_status generic_b_half(hyb_grid* g, void* const Bh[3]) {
    using C = cplx<T>;
    const ModeTables<T>& t = tables<T>(g);
    const int nk = g->nk;
    const int64_t rows = g->rows;
    C* spec = reinterpret_cast<C*>(g->spec);
    C* out = spec + 6 * rows * nk;
    const T a2 = (T)(g->d.dt / g->d.dx2);
    const T a3 = (T)(g->d.dims == 3 ? g->d.dt / g->d.dx3 : 0.0);
    const dim3 mgrid((unsigned)((int64_t)g->d.n3 * ((g->d.n2 + kModeRows - 1) / kModeRows) * ((nk + 31) / 32))), mblk(32, kModeRows);
    if (g->d.dims == 3) k_faraday_half<T, true><<<mgrid, mblk, 0, g->stream>>>(spec, out, nk, g->d.n2, g->d.n3, rows, t.S, a2, a3);
    else k_faraday_half<T, false><<<mgrid, mblk, 0, g->stream>>>(spec, out, nk, g->d.n2, 1, rows, t.S, a2, a3);
    HYB_CUDA_TRY(cudaGetLastError());
    RowPtrsW fout{};
    for (int c = 0; c < 3; c++) fout.p[c] = Bh[c];
    HYB_CUDA_TRY((launch_irfft<T, T>(out, 0, fout, 3, g->d.n1, rows, t, g->stream)));
    return HYB_OK;
}

template hyb_status generic_resident_import<float>(hyb_grid*);
template hyb_status generic_resident_import<double>(hyb_grid*);
template hyb_status generic_b_half<float>(hyb_grid*, void* const*);
template hyb_status generic_b_half<double>(hyb_grid*, void* const*);

int generic_launches_per_step(const hyb_grid* g) { return (amp_fused(g) || g->d.dims == 20) ? 3 : 4; }

template hyb_status generic_advance<float>(hyb_grid*, int);
template hyb_status generic_advance<double>(hyb_grid*, int);
template hyb_status generic_process_current<float>(hyb_grid*, bool, bool);
template hyb_status generic_process_current<double>(hyb_grid*, bool, bool);

}  // namespace hyb
