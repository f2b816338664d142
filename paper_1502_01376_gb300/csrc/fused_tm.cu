// fused_tm.cu -- the n1 = 4096 fused FP32 advance (body and design in tm_body.cuh): its kernel,
// the self-test kernel of the bounded waits, and the host side.
#include <vector>

#include "tm_body.cuh"

namespace hyb {

__global__ void __launch_bounds__(tmk::NT, 1) k_fused_tm(FusedBatch fb) {
    extern __shared__ __align__(128) unsigned char sm[];
    tm_body(fb, (int)blockIdx.x, (int)gridDim.x, sm);
}

// ------------------------------------------------------------------ self-test of the bounded waits
// which = 0: the release/acquire flag wait of the halo exchange, on a flag nothing sets;
// which = 1: the mbarrier wait of the row staging, on a phase nothing completes.
// Both must give up after `limit` cycles and report through *err.
__global__ void k_wait_probe(const int* flag, int* err, long long limit, int which) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    if (which == 0) {
        wait_flag(flag, 1, err, limit);
    } else {
        mbar_init(smem_addr(&bar), 1);
        mbar_fence_init();
        abort_flag = 0;
        mbar_wait(smem_addr(&bar), 0, err, &abort_flag, limit);
    }
}

cudaError_t wait_probe(int* dflag, int* derr, long long limit, int which, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(dflag, derr, limit, which);
    return cudaGetLastError();
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
