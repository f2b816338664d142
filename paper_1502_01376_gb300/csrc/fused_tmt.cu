// fused_tmt.cu -- the n1 = 512, 1024, 2048 fused FP32 advance (body and design in
// tmt_body.cuh): its kernel and the host side.
#include <algorithm>

#include "tmt_body.cuh"

namespace hyb {

template <int T>
__global__ void __launch_bounds__(384, 2) k_fused_tmt(FusedBatch fb) {
    extern __shared__ __align__(128) unsigned char sm[];
    tmt_body<T, false>(fb, (int)blockIdx.x, (int)gridDim.x, (int)threadIdx.x, sm, 0, 0u);
}

// ------------------------------------------------------------------ host side
template <int T>
static size_t tmt_smem() { return (size_t)Tmt<T>::SMEM; }

size_t fused_tmt_smem_bytes(int n1) {
    switch (n1) {
    case 512: return tmt_smem<32>();
    case 1024: return tmt_smem<64>();
    default: return tmt_smem<128>();
    }
}

template <int T>
static cudaError_t tmt_occ(int* units) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_tmt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tmt<T>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fused_tmt<T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    // CTAs per SM from the kernel's registers (warps take them in units of 256) and shared memory,
    // and at most two (the 512 TMEM columns of an SM); the runtime's occupancy query answers one
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_fused_tmt<T>);
    if (e != cudaSuccess) return e;
    int dev = 0, smem_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int occ_r = 65536 / (regs_warp * (Tmt<T>::NT / 32));
    const int occ_s = smem_sm / (Tmt<T>::SMEM + (int)fa.sharedSizeBytes + 1024);
    const int occ = std::max(1, std::min(std::min(occ_r, occ_s), 2));
    *units = occ * Tmt<T>::NTM;
    return cudaSuccess;
}

// work units (strips processed at once) per SM: CTAs per SM times teams per CTA
cudaError_t fused_tmt_occupancy(int n1, int* units) {
    switch (n1) {
    case 512: return tmt_occ<32>(units);
    case 1024: return tmt_occ<64>(units);
    default: return tmt_occ<128>(units);
    }
}

template <int T>
static cudaError_t tmt_launch(const FusedBatch& fb, int units, cudaStream_t s) {
    const int grid = (units + Tmt<T>::NTM - 1) / Tmt<T>::NTM;
    if (fb.flags) {          // every strip's team resident at once: cooperative launch
        void* args[] = {const_cast<FusedBatch*>(&fb)};
        return cudaLaunchCooperativeKernel((const void*)k_fused_tmt<T>, dim3(grid), dim3(Tmt<T>::NT), args, Tmt<T>::SMEM, s);
    }
    k_fused_tmt<T><<<grid, Tmt<T>::NT, Tmt<T>::SMEM, s>>>(fb);
    return cudaGetLastError();
}

// units: strips processed at once (at most CTAs x teams of the device)
cudaError_t fused_tmt_launch(int n1, const FusedBatch& fb, int units, cudaStream_t s) {
    switch (n1) {
    case 512: return tmt_launch<32>(fb, units, s);
    case 1024: return tmt_launch<64>(fb, units, s);
    default: return tmt_launch<128>(fb, units, s);
    }
}

}  // namespace hyb
