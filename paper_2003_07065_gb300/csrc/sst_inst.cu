// Instantiates the NF-templated kernels for one DFT length (SST_NF, set on
// the compiler command line) and exports their launcher table.
#include "sst_kernels.cuh"
#include "sst_launch.h"

#ifndef SST_NF
#error "compile with -DSST_NF=<power of two in [64, 8192]>"
#endif

namespace sst {
namespace {

constexpr int NF = SST_NF;
using C = Cfg<NF>;

const void *kernel_of(int kind) {
    switch (kind) {
        case KIND_ABSMAX: return (const void *)k_absmax<NF>;
        case KIND_FWD_T: return (const void *)k_forward<NF, MODE_T>;
        case KIND_FWD_STFT: return (const void *)k_forward<NF, MODE_STFT>;
        case KIND_FWD_MAP: return (const void *)k_forward<NF, MODE_MAP>;
        case KIND_FWD_SPEC: return (const void *)k_forward<NF, MODE_SPEC>;
        case KIND_INV: return (const void *)k_inverse<NF, true>;
        case KIND_INV_WIDE: return (const void *)k_inverse<NF, false>;
        case KIND_B_ABSMAX: return (const void *)k_absmax_batch<NF>;
        case KIND_B_FWD: return (const void *)k_forward_batch<NF>;
        case KIND_B_INV: return (const void *)k_inverse_batch<NF, true>;
        case KIND_B_INV_WIDE: return (const void *)k_inverse_batch<NF, false>;
    }
    return nullptr;
}

cudaError_t set_smem(int kind, size_t bytes) {
    const void *k = kernel_of(kind);
    if (!k) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t occupancy(int kind, size_t bytes, int *blocks) {
    const void *k = kernel_of(kind);
    if (!k) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, C::TPF, bytes);
}

cudaError_t absmax(const SstDev &d, const float *x, float *partial, int grid, size_t smem, cudaStream_t st) {
    k_absmax<NF><<<grid, C::TPF, smem, st>>>(d, x, partial);
    return cudaGetLastError();
}

cudaError_t forward(const SstDev &d, int kind, const float *x, const SstScalars *sc, void *out0, void *out1,
                    int grid, size_t smem, cudaStream_t st) {
    switch (kind) {
        case KIND_FWD_T:
            k_forward<NF, MODE_T><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        case KIND_FWD_STFT:
            k_forward<NF, MODE_STFT><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        case KIND_FWD_MAP:
            k_forward<NF, MODE_MAP><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        case KIND_FWD_SPEC:
            k_forward<NF, MODE_SPEC><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t inverse(const SstDev &d, int kind, const float2 *T, float *partial, size_t smem, cudaStream_t st) {
    if (kind == KIND_INV)
        k_inverse<NF, true><<<(unsigned)d.ntiles, C::TPF, smem, st>>>(d, T, partial);
    else if (kind == KIND_INV_WIDE)
        k_inverse<NF, false><<<(unsigned)d.ntiles, C::TPF, smem, st>>>(d, T, partial);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t batch(int kind, const BatchChan *ch, const BatchItem *items, int nitems, int max_nbo, int grid,
                  size_t smem, float *partial, cudaStream_t st) {
    switch (kind) {
        case KIND_B_ABSMAX: k_absmax_batch<NF><<<grid, C::TPF, smem, st>>>(ch, items, nitems, partial); break;
        case KIND_B_FWD: k_forward_batch<NF><<<grid, C::TPF, smem, st>>>(ch, items, nitems, max_nbo); break;
        case KIND_B_INV: k_inverse_batch<NF, true><<<grid, C::TPF, smem, st>>>(ch, items, nitems); break;
        case KIND_B_INV_WIDE: k_inverse_batch<NF, false><<<grid, C::TPF, smem, st>>>(ch, items, nitems); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

const KernelTable table = {NF, C::TPF, (size_t)C::BUF * sizeof(float2) + 128, set_smem, occupancy,
                           absmax, forward, inverse, batch};

}  // namespace

#define SST_CAT2(a, b) a##b
#define SST_CAT(a, b) SST_CAT2(a, b)
const KernelTable *SST_CAT(table_nf_, SST_NF)() { return &table; }

}  // namespace sst
