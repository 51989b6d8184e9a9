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

constexpr int CLS1 = cls_for<NF>(1), CLS2 = cls_for<NF>(2);

int cls_of(int kind) { return kind >> KIND_CLS_SHIFT; }

// the forward with aliased accumulators exists for classes 1 and 2 only
template <int MODE> const void *forward_alias_kernel(int cls) {
    if constexpr (CLS1 > 0 && CLS2 > 0) {
        if (cls == 1) return (const void *)k_forward_alias<NF, MODE, CLS1>;
        if (cls == 2) return (const void *)k_forward_alias<NF, MODE, CLS2>;
    }
    return nullptr;
}

template <int MODE>
bool launch_forward_alias(int cls, const SstDev &d, const float *x, const SstScalars *sc, void *out0, int grid,
                          size_t smem, cudaStream_t st) {
    if constexpr (CLS1 > 0 && CLS2 > 0) {
        if (cls == 1) {
            k_forward_alias<NF, MODE, CLS1><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, nullptr);
            return true;
        }
        if (cls == 2) {
            k_forward_alias<NF, MODE, CLS2><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, nullptr);
            return true;
        }
    }
    return false;
}

template <int MODE> const void *forward_kernel(int cls) {
    if (cls == 1) return (const void *)k_forward<NF, MODE, CLS1>;
    if (cls == 2) return (const void *)k_forward<NF, MODE, CLS2>;
    return (const void *)k_forward<NF, MODE, 0>;
}

const void *kernel_of(int kind) {
    const int cls = cls_of(kind);
    switch (kind & ((1 << KIND_CLS_SHIFT) - 1)) {
        case KIND_ABSMAX:
            if (cls == 1) return (const void *)k_absmax<NF, CLS1>;
            if (cls == 2) return (const void *)k_absmax<NF, CLS2>;
            return (const void *)k_absmax<NF>;
        case KIND_FWD_T: return forward_kernel<MODE_T>(cls);
        case KIND_FWD_STFT: return (const void *)k_forward<NF, MODE_STFT>;
        case KIND_FWD_MAP: return (const void *)k_forward<NF, MODE_MAP>;
        case KIND_FWD_SPEC: return forward_kernel<MODE_SPEC>(cls);
        case KIND_FWD_SO_T: return (const void *)k_forward_so<NF, MODE_T>;
        case KIND_FWD_SO_MAP: return (const void *)k_forward_so<NF, MODE_MAP>;
        case KIND_FWD_TA: return forward_alias_kernel<MODE_T>(cls);
        case KIND_FWD_SPECA: return forward_alias_kernel<MODE_SPEC>(cls);
        case KIND_INV:
            if (cls == 1) return (const void *)k_inverse<NF, true, CLS1>;
            if (cls == 2) return (const void *)k_inverse<NF, true, CLS2>;
            return (const void *)k_inverse<NF, true>;
        case KIND_INV_WIDE: return (const void *)k_inverse<NF, false>;
        case KIND_INV_LONG: return (const void *)k_inverse<NF, false, CLS_LONG>;
        case KIND_FUSED:
            if (cls == 1) return (const void *)k_fused<NF, true, CLS1>;
            if (cls == 2) return (const void *)k_fused<NF, true, CLS2>;
            return (const void *)k_fused<NF, true, 0>;
        case KIND_FUSED_WIDE: return (const void *)k_fused<NF, false, 0>;
        case KIND_FUSED_LONG: return (const void *)k_fused<NF, false, CLS_LONG>;
        case KIND_B_ABSMAX: return (const void *)k_absmax_batch<NF>;
        case KIND_B_FWD:
            if (cls == 1) return (const void *)k_forward_batch<NF, CLS1>;
            if (cls == 2) return (const void *)k_forward_batch<NF, CLS2>;
            return (const void *)k_forward_batch<NF>;
        case KIND_B_INV:
            if (cls == 1) return (const void *)k_inverse_batch<NF, true, CLS1>;
            if (cls == 2) return (const void *)k_inverse_batch<NF, true, CLS2>;
            return (const void *)k_inverse_batch<NF, true>;
        case KIND_B_INV_WIDE: return (const void *)k_inverse_batch<NF, false>;
        case KIND_B_INV_LONG: return (const void *)k_inverse_batch<NF, false, CLS_LONG>;
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

cudaError_t absmax(const SstDev &d, int cls, const float *x, float *partial, int grid, size_t smem, cudaStream_t st) {
    if (cls == 1) k_absmax<NF, CLS1><<<grid, C::TPF, smem, st>>>(d, x, partial);
    else if (cls == 2) k_absmax<NF, CLS2><<<grid, C::TPF, smem, st>>>(d, x, partial);
    else k_absmax<NF><<<grid, C::TPF, smem, st>>>(d, x, partial);
    return cudaGetLastError();
}

template <int MODE>
void launch_forward(int cls, const SstDev &d, const float *x, const SstScalars *sc, void *out0, void *out1, int grid,
                    size_t smem, cudaStream_t st) {
    if (cls == 1) k_forward<NF, MODE, CLS1><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
    else if (cls == 2) k_forward<NF, MODE, CLS2><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
    else k_forward<NF, MODE, 0><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
}

cudaError_t forward(const SstDev &d, int kind, const float *x, const SstScalars *sc, void *out0, void *out1,
                    int grid, size_t smem, cudaStream_t st) {
    const int cls = cls_of(kind);
    switch (kind & ((1 << KIND_CLS_SHIFT) - 1)) {
        case KIND_FWD_T:
            launch_forward<MODE_T>(cls, d, x, sc, out0, out1, grid, smem, st);
            break;
        case KIND_FWD_STFT:
            k_forward<NF, MODE_STFT><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        case KIND_FWD_MAP:
            k_forward<NF, MODE_MAP><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        case KIND_FWD_SPEC:
            launch_forward<MODE_SPEC>(cls, d, x, sc, out0, out1, grid, smem, st);
            break;
        case KIND_FWD_SO_T:
            k_forward_so<NF, MODE_T><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        case KIND_FWD_SO_MAP:
            k_forward_so<NF, MODE_MAP><<<grid, C::TPF, smem, st>>>(d, x, sc, (float2 *)out0, out1);
            break;
        case KIND_FWD_TA:
            if (!launch_forward_alias<MODE_T>(cls, d, x, sc, out0, grid, smem, st)) return cudaErrorInvalidValue;
            break;
        case KIND_FWD_SPECA:
            if (!launch_forward_alias<MODE_SPEC>(cls, d, x, sc, out0, grid, smem, st)) return cudaErrorInvalidValue;
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t inverse(const SstDev &d, int kind, const float2 *T, float *partial, size_t smem, cudaStream_t st) {
    const unsigned grid = (unsigned)d.ntiles;
    if (kind == kind_cls(KIND_INV, 1))
        k_inverse<NF, true, CLS1><<<grid, C::TPF, smem, st>>>(d, T, partial);
    else if (kind == kind_cls(KIND_INV, 2))
        k_inverse<NF, true, CLS2><<<grid, C::TPF, smem, st>>>(d, T, partial);
    else if (kind == KIND_INV)
        k_inverse<NF, true><<<(unsigned)d.ntiles, C::TPF, smem, st>>>(d, T, partial);
    else if (kind == KIND_INV_WIDE)
        k_inverse<NF, false><<<(unsigned)d.ntiles, C::TPF, smem, st>>>(d, T, partial);
    else if (kind == KIND_INV_LONG)
        k_inverse<NF, false, CLS_LONG><<<grid, C::TPF, smem, st>>>(d, T, partial);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t fused(const SstDev &d, int kind, const float *x, const SstScalars *sc, float *partial, size_t smem,
                  cudaStream_t st) {
    const unsigned grid = (unsigned)d.ntiles;
    if (kind == kind_cls(KIND_FUSED, 1))
        k_fused<NF, true, CLS1><<<grid, C::TPF, smem, st>>>(d, x, sc, partial);
    else if (kind == kind_cls(KIND_FUSED, 2))
        k_fused<NF, true, CLS2><<<grid, C::TPF, smem, st>>>(d, x, sc, partial);
    else if (kind == KIND_FUSED)
        k_fused<NF, true, 0><<<grid, C::TPF, smem, st>>>(d, x, sc, partial);
    else if (kind == KIND_FUSED_WIDE)
        k_fused<NF, false, 0><<<grid, C::TPF, smem, st>>>(d, x, sc, partial);
    else if (kind == KIND_FUSED_LONG)
        k_fused<NF, false, CLS_LONG><<<grid, C::TPF, smem, st>>>(d, x, sc, partial);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t batch(int kind, const BatchChan *ch, const BatchItem *items, int nitems, int max_nbo, int grid,
                  size_t smem, float *partial, cudaStream_t st) {
    const int cls = cls_of(kind);
    switch (kind & ((1 << KIND_CLS_SHIFT) - 1)) {
        case KIND_B_ABSMAX: k_absmax_batch<NF><<<grid, C::TPF, smem, st>>>(ch, items, nitems, partial); break;
        case KIND_B_FWD:
            if (cls == 1) k_forward_batch<NF, CLS1><<<grid, C::TPF, smem, st>>>(ch, items, nitems, max_nbo);
            else if (cls == 2) k_forward_batch<NF, CLS2><<<grid, C::TPF, smem, st>>>(ch, items, nitems, max_nbo);
            else k_forward_batch<NF><<<grid, C::TPF, smem, st>>>(ch, items, nitems, max_nbo);
            break;
        case KIND_B_INV:
            if (cls == 1) k_inverse_batch<NF, true, CLS1><<<grid, C::TPF, smem, st>>>(ch, items, nitems);
            else if (cls == 2) k_inverse_batch<NF, true, CLS2><<<grid, C::TPF, smem, st>>>(ch, items, nitems);
            else k_inverse_batch<NF, true><<<grid, C::TPF, smem, st>>>(ch, items, nitems);
            break;
        case KIND_B_INV_WIDE: k_inverse_batch<NF, false><<<grid, C::TPF, smem, st>>>(ch, items, nitems); break;
        case KIND_B_INV_LONG: k_inverse_batch<NF, false, CLS_LONG><<<grid, C::TPF, smem, st>>>(ch, items, nitems); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

const KernelTable table = {NF, C::R1, C::TPF, (size_t)C::BUF * sizeof(float2) + 128, set_smem, occupancy,
                           absmax, forward, inverse, fused, batch};

}  // namespace

#define SST_CAT2(a, b) a##b
#define SST_CAT(a, b) SST_CAT2(a, b)
const KernelTable *SST_CAT(table_nf_, SST_NF)() { return &table; }

}  // namespace sst
