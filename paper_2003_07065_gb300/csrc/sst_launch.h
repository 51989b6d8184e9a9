// Per-NF launcher table: every NF-templated kernel is instantiated in its own
// translation unit (sst_inst.cu compiled once per NF) and reached through
// this table, so the host code needs no templates.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "sst_dev.h"

namespace sst {

enum { KIND_ABSMAX = 0, KIND_FWD_T = 1, KIND_FWD_STFT = 2, KIND_FWD_MAP = 3, KIND_INV = 4, KIND_INV_WIDE = 5,
       KIND_B_ABSMAX = 6, KIND_B_FWD = 7, KIND_B_INV = 8, KIND_B_INV_WIDE = 9, KIND_FWD_SPEC = 10,
       KIND_FUSED = 11, KIND_FUSED_WIDE = 12, KIND_FWD_TA = 13, KIND_FWD_SPECA = 14, KIND_FWD_SO_T = 15,
       KIND_FWD_SO_MAP = 16, KIND_INV_LONG = 17, KIND_FUSED_LONG = 18, KIND_B_INV_LONG = 19, KIND_COUNT = 20 };
// KIND_*_LONG: a window longer than nf + 1 (the inverse, fused and batched
// inverse kernels of class CLS_LONG).
// KIND_FWD_SO_T / KIND_FWD_SO_MAP: the second-order forward (k_forward_so).
// KIND_FWD_TA / KIND_FWD_SPECA: the forward with its accumulators in the frame
// buffer (k_forward_alias), pruning classes 1 and 2 only.

// A forward (KIND_FWD_T, KIND_FWD_SPEC), inverse (KIND_INV) or fused
// forward + inverse (KIND_FUSED) kind may carry a
// pruning class (band_class, 1 or 2) in the bits from KIND_CLS_SHIFT up;
// tables whose first radix is not 16 run class 0 for every class.
constexpr int KIND_CLS_SHIFT = 8;
inline int kind_cls(int kind, int cls) { return kind | (cls << KIND_CLS_SHIFT); }

struct KernelTable {
    int nf;
    int r1;              // radix of the first FFT pass
    int tpf;             // threads per CTA
    size_t smem_frame;   // bytes of the padded frame buffer plus reduction scratch
    // raise the dynamic shared-memory limit of a kernel kind
    cudaError_t (*set_smem)(int kind, size_t bytes);
    // resident CTAs per SM for a kernel kind at a dynamic shared-memory size
    cudaError_t (*occupancy)(int kind, size_t bytes, int *blocks);
    // the max |S^g|^2 pre-pass; cls: the plan's pruning class (0 for any plan)
    cudaError_t (*absmax)(const SstDev &d, int cls, const float *x, float *partial, int grid, size_t smem,
                          cudaStream_t st);
    cudaError_t (*forward)(const SstDev &d, int kind, const float *x, const SstScalars *sc, void *out0,
                           void *out1, int grid, size_t smem, cudaStream_t st);
    // kind: KIND_INV (window L <= nf/2 + 1), KIND_INV_WIDE (L <= nf + 1) or KIND_INV_LONG
    cudaError_t (*inverse)(const SstDev &d, int kind, const float2 *T, float *partial, size_t smem, cudaStream_t st);
    // fused forward + inverse over the plan's inverse tiles (kind: KIND_FUSED
    // with its class, KIND_FUSED_WIDE or KIND_FUSED_LONG); partial is the overlap-add buffer
    cudaError_t (*fused)(const SstDev &d, int kind, const float *x, const SstScalars *sc, float *partial,
                         size_t smem, cudaStream_t st);
    // batched kernels over a work-item table (kind: KIND_B_*)
    cudaError_t (*batch)(int kind, const BatchChan *ch, const BatchItem *items, int nitems, int max_nbo, int grid,
                         size_t smem, float *partial, cudaStream_t st);
};

const KernelTable *table_for_nf(int nf);

}  // namespace sst
