// batch_step.cu -- the batched step (many fused 2D grids of uneven sizes plus quasi-3D modes) as
// ONE persistent cooperative launch of 768-thread CTAs, one per SM.  The CTAs are split into
// roles by ranges of blockIdx.x, in proportions the batch autotuner sets:
//
//   * a 2D group (all fused grids with one n1) first copies the halo rows of its work items (one
//     warp per row), meets at a barrier of the role's CTAs, then sweeps its work items: n1 = 4096
//     with the 768-thread body of the single-grid kernel (three groups of 256, 512 TMEM columns);
//     n1 = 512 .. 2048 with two 384-thread team bodies per CTA, each half with its own 256 TMEM
//     columns, shared memory and named barriers;
//   * the quasi-3D modes run their three stages (z transform of the nine arrays of every mode,
//     leapfrog, inverse z transform of the six advanced spectra) as three 256-thread parts per CTA,
//     with a barrier of the role's CTAs between the stages.
//
// Role barriers are counters in global memory with a generation word, so that they need no reset
// between steps (the launch is replayed from a CUDA graph); every wait is bounded and reports
// through the role's error word.  The roles share no data: a step is the same arithmetic, in the
// same order per output, as the separate launches of batch.cu's graph, and gives the same bits.
#include <algorithm>

#include "batch_step.cuh"
#include "tm_body.cuh"
#include "tmt_body.cuh"

namespace hyb {

namespace {
constexpr int kStepThreads = 768;
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kQ3Part = (kQ2kA + kQ2kB + kQ2k) * 8;                // exchange buffers and staging row of a part
constexpr int kTeamBytes = cmax(cmax(2 * Tmt<32>::SMEM_MEGA, 2 * Tmt<64>::SMEM_MEGA), 2 * Tmt<128>::SMEM_MEGA);
constexpr int kQ3Bar = 3 * kQ3Part + kQ2kTw * 8;                    // quasi-3D role: 12 mbarriers, 3 abort flags
constexpr int kStepSmem = cmax(cmax(tmk::SMEM, kTeamBytes + 16), kQ3Bar + 12 * 8 + 3 * 4);
static_assert(2 * 9 * 256 * 8 <= kQ3Part, "the leapfrog's two stages fit a part's transform buffers");
}  // namespace

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// barrier of the ncta CTAs of one role: s[0] counts arrivals, s[1] is the generation.  The last CTA
// to arrive resets the count and then advances the generation; the others wait for the generation
// they saw before arriving to change (bounded: after `limit` cycles, about 2 s by default, bit 1 of
// *err is set and the CTA goes on).  Global writes of the CTA before the barrier are visible to the
// role's CTAs after it.
__device__ __forceinline__ void role_sync(unsigned* s, int ncta, int* err, long long limit = kWaitCycles) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = s + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(s, 1u) == (unsigned)ncta - 1) {
            atomicExch(s, 0u);
            __threadfence();
            atomicAdd(s + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > limit) { if (err) atomicOr(err, 2); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// the quasi-3D modes on CTA vb of the role's n CTAs: three 256-thread parts per CTA.  The CTA's
// shared memory holds each part's exchange buffers and staging row (filled by bulk copy) and the z
// transform's twiddle table: the L1 left beside the 2D roles' shared memory is small, and a part
// has no registers to spare for holding the next row.  The leapfrog sweeps columns: a part takes
// one (mode, block of 256 axial modes, chunk of radial rows), the chunks cut so that the columns
// are at most as many as the parts (one round); its rows arrive by bulk copy into the part's
// transform buffers, which the leapfrog does not otherwise use.  Spectra written by one stage are
// read by bulk copy in the next: a proxy fence follows each role barrier.
__device__ __forceinline__ void q3_role(const StepArgs& a, int vb, unsigned char* sm) {
    const int part = threadIdx.x >> 8, t = threadIdx.x & 255;
    const int n = a.q3_ncta, parts = 3 * n;
    const Q3Args& q = a.q3;
    float2* bufA = reinterpret_cast<float2*>(sm + part * kQ3Part);
    float2* bufB = bufA + kQ2kA;
    float2* tws = reinterpret_cast<float2*>(sm + 3 * kQ3Part);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kQ3Bar);
    volatile int* aborts = reinterpret_cast<volatile int*>(sm + kQ3Bar + 12 * 8);
    for (int i = threadIdx.x; i < kQ2kTw; i += blockDim.x) tws[i] = q.tw2k[i];
    if (t == 0) {
        for (int b = 0; b < 4; b++) mbar_init(smem_addr(bars + 4 * part + b), 1);
        aborts[part] = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const QStage fwd{bufB + kQ2kB, smem_addr(bars + 4 * part), a.q3_err, aborts + part};
    const QStage inv{bufB + kQ2kB, smem_addr(bars + 4 * part + 1), a.q3_err, aborts + part};
    const uint32_t lbar0 = smem_addr(bars + 4 * part + 2), lbar1 = smem_addr(bars + 4 * part + 3);
    uint32_t lph = 0;
    cfft2048_body<false, true>(q.fin, q.nr, 9, tws, 3 * vb + part, parts, t, bufA, bufB, 1 + part, fwd);
    role_sync(a.sync + 2 * kRoleQ3, n, a.q3_err);
    asm volatile("fence.proxy.async.global;" ::: "memory");
    constexpr int nkb = kQ2k / 256;                                 // blocks of 256 axial modes per row
    const int ncol = nkb * q.nm;
    const int nch = max(1, min(q.nr, parts / ncol));                // row chunks per column
    const int rows = (q.nr + nch - 1) / nch;
    for (int u = 3 * vb + part; u < ncol * nch; u += parts) {
        const int col = u % ncol, ch = u / ncol;
        const int j0 = ch * rows, j1 = min(q.nr, j0 + rows);
        if (j0 < j1)
            qleap_column<float>(q.ql, kQ2k, q.nr, q.dr, col % nkb, col / nkb, j0, j1, t, bufA, lbar0, lbar1, lph, 1 + part,
                                a.q3_err, aborts + part);
    }
    // after a wait that gave up, the stages still in flight land before the buffers are reused
    if (aborts[part] && t == 0) {
        if (lph & 4u) mbar_drain(lbar0, (lph & 1u) ^ 1u);
        if (lph & 8u) mbar_drain(lbar1, ((lph >> 1) & 1u) ^ 1u);
    }
    role_sync(a.sync + 2 * kRoleQ3, n, a.q3_err);
    asm volatile("fence.proxy.async.global;" ::: "memory");
    cfft2048_body<true, true>(q.fout, q.nr, 6, tws, 3 * vb + part, parts, t, bufA, bufB, 1 + part, inv);
}

__global__ void __launch_bounds__(kStepThreads, 1) k_batch_step(const __grid_constant__ StepArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int cta = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned long long t_start = 0;
    if (a.stamp && tid == 0) t_start = gtimer();
    int role = -1;
#pragma unroll
    for (int r = 0; r < 4; r++)
        if (cta >= a.r2[r].cta0 && cta < a.r2[r].cta0 + a.r2[r].ncta) role = r;
    if (role < 0 && cta >= a.q3_cta0 && cta < a.q3_cta0 + a.q3_ncta) role = kRoleQ3;
    if (role < 0) return;
    if (role == kRoleQ3) {
        q3_role(a, cta - a.q3_cta0, sm);
    } else {
        const StepRole2D& R = a.r2[role];
        const int vb = cta - R.cta0;
        constexpr int kWarps = kStepThreads / 32;
        for (int w = vb * kWarps + warp; w < R.n_halo; w += R.ncta * kWarps) copy_row_warp(R.halo[w], lane);
        role_sync(a.sync + 2 * role, R.ncta, R.fb.err);
        // the halo rows were written through the generic proxy; the bodies may read them by bulk copy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (role == kRoleTM) {
            tm_body(R.fb, vb, R.ncta, sm);
        } else {
            uint32_t* s_t = reinterpret_cast<uint32_t*>(sm + kTeamBytes);
            if (warp == 0) {
                tm_alloc(smem_addr(s_t), 512);
                tm_relinquish();
            }
            tm_fence_before();
            __syncthreads();
            tm_fence_after();
            const uint32_t tb = *s_t;
            const int half = tid >= 384 ? 1 : 0, ht = tid - 384 * half;
            const uint32_t th = tb + 256u * (uint32_t)half;
            if (role == kRoleT32)
                tmt_body<32, true>(R.fb, 2 * vb + half, 2 * R.ncta, ht, sm + half * Tmt<32>::SMEM_MEGA, half, th);
            else if (role == kRoleT64)
                tmt_body<64, true>(R.fb, 2 * vb + half, 2 * R.ncta, ht, sm + half * Tmt<64>::SMEM_MEGA, half, th);
            else
                tmt_body<128, true>(R.fb, 2 * vb + half, 2 * R.ncta, ht, sm + half * Tmt<128>::SMEM_MEGA, half, th);
            tm_fence_before();
            __syncthreads();
            tm_fence_after();
            if (warp == 0) tm_dealloc(tb, 512);
        }
    }
    if (a.stamp && tid == 0) {
        atomicMin(a.stamp + 2 * role, t_start);
        atomicMax(a.stamp + 2 * role + 1, gtimer());
    }
}

// self-test of the role barrier: a role of two CTAs of which only this one arrives; the wait must
// give up after `limit` cycles and report through *err
__global__ void k_role_probe(unsigned* s, int* err, long long limit) { role_sync(s, 2, err, limit); }

// ------------------------------------------------------------------ host side
size_t batch_step_smem_bytes() { return (size_t)kStepSmem; }

cudaError_t batch_step_ctas(int* n) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_step, kStepThreads, kStepSmem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *n = occ >= 1 ? sms : 0;           // one CTA per SM (TMEM: 512 columns per CTA)
    return cudaSuccess;
}

cudaError_t role_probe(unsigned* sync, int* err, long long limit, cudaStream_t s) {
    k_role_probe<<<1, 32, 0, s>>>(sync, err, limit);
    return cudaGetLastError();
}

cudaError_t batch_step_launch(const StepArgs& a, int grid, cudaStream_t s) {
    void* args[] = {const_cast<StepArgs*>(&a)};
    return cudaLaunchCooperativeKernel((const void*)k_batch_step, dim3(grid), dim3(kStepThreads), args, kStepSmem, s);
}

}  // namespace hyb
