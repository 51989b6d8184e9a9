// Internal declarations shared by the host translation units of libsst.so
// (plan object, error reporting, launch accounting, per-kernel profiling).
#pragma once
#include <atomic>
#include <cstdint>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sst.h"
#include "sst_dev.h"
#include "sst_launch.h"

#define SST_API extern "C" __attribute__((visibility("default")))
// helpers of libsst.so that the tensor-form library (libsst_tc.so, linked
// against it) calls too, so both share one error message, launch counter
// and profile record
#define SST_SHARED __attribute__((visibility("default")))

namespace sst {

// An NVTX range over one C-ABI call, named as the call, for timeline tools
// (Nsight Systems); NVTX does nothing unless such a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define SST_NVTX_RANGE() ::sst::NvtxRange sst_nvtx_range_(__func__)

// error reporting: sets the thread-local message returned by sst_last_error
SST_SHARED sst_status fail(sst_status s, const char *fmt, ...);
SST_SHARED sst_status cuda_fail(cudaError_t e, const char *what);
SST_SHARED void count_launch();
// raise (never lower) a kernel's dynamic shared-memory limit, so plans,
// batches and streams with different needs can share the kernels
cudaError_t raise_smem(const KernelTable *kt, int kind, size_t bytes);
// launchers of two small kernels of libsst.so (k_absx: max |x| per CTA into
// partial[0, grid); k_gamma: the call scalars from pre-pass partials)
SST_SHARED cudaError_t launch_absx(const float *x, int64_t n, float *partial, int grid, cudaStream_t st);
SST_SHARED cudaError_t launch_gamma(const float *partial, int count, float frac2, int from_x, float bound_mul,
                                    int log2_nb, SstScalars *sc, float *maxv_out, const unsigned *gate,
                                    cudaStream_t st);

#define SST_CU(call, what)                                      \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::sst::cuda_fail(e_, what); \
    } while (0)

// per-kernel timing (sst_profile_enable): events around each launch
enum { PK_ABSMAX = 0, PK_GAMMA, PK_FORWARD, PK_STFT, PK_MAP, PK_INVERSE, PK_FINALIZE, PK_OTHER, PK_FUSED };
SST_SHARED bool profiling_on();
SST_SHARED void profile_record(int kind, cudaEvent_t a, cudaEvent_t b);

struct ProfScope {
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(int k, cudaStream_t s) : kind(k), st(s) {
        if (profiling_on()) {
            if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) cudaEventRecord(a, st);
            else a = b = nullptr;
        }
    }
    void done() {
        if (a && b) {
            cudaEventRecord(b, st);
            profile_record(kind, a, b);
            a = b = nullptr;
        }
    }
    ~ProfScope() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

#define SST_LAUNCHED_K(kind, st, call, what)                      \
    do {                                                          \
        ::sst::ProfScope ps_(kind, st);                           \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::sst::cuda_fail(e_, what); \
        ps_.done();                                               \
        ::sst::count_launch();                                    \
    } while (0)

}  // namespace sst

// ------------------------------------------------------------ plan
struct sst_plan {
    sst_params p;
    int device = 0;
    int num_sms = 0;
    sst::SstDev d;
    const sst::KernelTable *kt = nullptr;
    void *dmem = nullptr;
    float gamma_frac2 = 0.f;
    float sum_abs_g = 0.f;   // bound factor |S^g| <= max|x| sum|g| (rounded up)
    size_t smem_fwd_t = 0, smem_fwd_x = 0, smem_absmax = 0, smem_inv = 0;
    int inv_kind = sst::KIND_INV;            // with its pruning class (kind_cls)
    int absmax_cls = 0;                      // pruning class of the max |S^g| pre-pass
    int kind_fwd_t = sst::KIND_FWD_T;
    int kind_fwd_spec = sst::KIND_FWD_SPEC;
    int grid_absmax = 0, grid_fwd = 0, grid_fwd_x = 0;
    // fused forward + inverse (sst_forward_inverse without a TFR): kind with
    // its class, shared memory, and whether it fits this device
    int kind_fused = sst::KIND_FUSED;
    size_t smem_fused = 0;
    bool fused_ok = false;
    size_t ws_bytes = 0, ws_off_partial = 0, ws_off_ola = 0;
    // one-pass relative threshold
    bool spec = false;
    size_t smem_fwd_spec = 0, ws_off_spec = 0;
    int grid_fwd_spec = 0, spec_tf = 1, spec_cap = 0;
    size_t smem_frame_absmax = 0;
    // one-pass threshold of the path without a TFR output (k_fused_settle)
    bool fused_spec = false;
    int fused_cap = 0;
    size_t ws_off_fused = 0;
    size_t smem_settle = 0;
    std::vector<double> g64, dgs64;   // FP64 window g and s g' (basis of the tensor form)
    bool custom_window = false;       // g was supplied by the caller (not the built-in Gaussian)
    std::atomic<int> test_withhold{0};      // one-shot test hook (sst_test_withhold_row_copy)
    std::atomic<int> test_withhold_fwd{0};  // one-shot test hook (sst_test_withhold_sample_copy)
};
