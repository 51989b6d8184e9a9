// Device-side view of a plan, passed to every kernel by value.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sst.h"

namespace sst {

// Records of the one-pass relative threshold (run_forward_spec in
// sst_capi.cu): sources whose keep/drop decision waits for the call's exact
// max |S^g|, and the fine bins they land in with the exact sums of the
// sources already kept there.
struct SpecSrc {
    int32_t bin;      // index of its SpecBin, or -1 when that record did not fit
    float vr, vi;     // S^g
    float mag2;       // |S^g|^2 as the forward kernel computed it
};
struct SpecBin {
    int64_t m;        // frame
    int32_t l;        // fine bin
    uint32_t w[4];    // exact sums (re lo, re hi, im lo, im hi), see tacc_*
    int32_t pad;
};
struct SpecBuf {
    unsigned *ctl;    // [0] max |S^g|^2 (float bits), [1] source records taken, [2] bin records taken,
                      // [3] overflow, [4] max_m A_m (float bits), [5] waiting sources, [6] their bins
    SpecSrc *src;
    SpecBin *bin;
    int cap_src, cap_bin;
};

struct SstDev {
    // tables (device pointers owned by the plan)
    const float2 *win;  // (g[j], g'[j]) for j = -M..M, L entries
    const float *g;     // g[j], L entries
    const float2 *tw;   // Stockham twiddles per pass, [4 (Ns - R1) / 15 + i Ns + k] = W_{16 Ns}^{2^i k}, i = 0..3
    // inverse sub-grid twiddle exp(+2 pi i s n / (z nf)) for the last-pass output slot
    // q = j + r nf/16 (n = q, or q - nf when wrapped) = twb[s nf/16 + j] * twc[(2 s + wrapped) 16 + r]
    const float2 *twb;  // [s nf/16 + j] = exp(2 pi i s j / (z nf))
    const float2 *twc;  // [(2 s + w) 16 + r] = exp(2 pi i s r / (16 z)) * (w ? exp(-2 pi i s / z) : 1)
    const float2 *twn;  // [s] = exp(-2 pi i s (nf/2) / (z nf)), for the tap n = -nf/2
    const float *rD_left;   // 1 / D[p] for p in [0, EL)
    const float *rD_per;    // 1 / D[p] for p in [EL, ER), indexed by p mod hop
    const float *rD_right;  // 1 / D[p] for p in [ER, n)
    int64_t n, F;
    int64_t EL, ER;
    int L, M, hop, nf, z;
    int k_lo, k_hi, nb, nbo;
    int log2_nb;        // ceil(log2(nb))
    float c_if;         // nf / (2 pi s): IF offset factor for the packed, scaled S^g'
    float dscale;       // 1 / s: the packed imaginary part carries s g' (s a power of two)
    // second-order IF (sst_forward2): windows (s2 g'', s3 t g) and (s4 t g', 0),
    // L entries each (null when the plan's window is not the built-in
    // Gaussian), and the exact inverse scales 1 / s2, 1 / s3, 1 / s4
    const float2 *win2, *win3;
    float r2, r3, r4;
    float c_so;         // nf / (2 pi): rad/sample -> bins
    float gamma2_abs;   // absolute threshold squared
    int relative;       // threshold from the pre-pass
    int B;              // frames per inverse tile (even)
    int seg_len;        // (B - 1) hop + L
    int64_t ntiles;
    // buffer placement (all zero for a whole-signal call); used by streams:
    int64_t xoff;       // the x pointer holds samples from global index xoff on
    int trow_cap;       // T row of frame m is m % trow_cap (ring), or m when 0
    int tile_cap;       // overlap-add slot of tile t is t % tile_cap, or t when 0
    // one-pass relative threshold (zero / null otherwise)
    const unsigned *gate;  // when set, the pre-pass and forward kernels run only if *gate != 0
    int sample_stride;     // pre-pass: every sample_stride-th group of four frames (0 or 1: all)
    SpecBuf spec;          // forward MODE_SPEC records
    // one-pass relative threshold of the path without a TFR output (k_fused;
    // null otherwise): per inverse tile, the sources between the two bounds
    // go to fused_rec[tile * fused_cap + i] (m, l, w = S^g re, im, |S^g|^2 as
    // float bits, source bin) and their count to fused_count[tile]
    SpecBin *fused_rec;
    int32_t *fused_count;
    int fused_cap;
    const float2 *twf;     // exp(2 pi i j / (z nf)), j in [0, z nf): the settling pass's phases
    // component recovery (sst_inverse_zone): when set, the inverse keeps only
    // the coefficients of output bins l with |l - zone[m]| <= zone_hw (none
    // where zone[m] < 0), the zone of Eq. 15
    const int32_t *zone;
    int zone_hw;
    // status word of the call (sst_check), or null: the inverse ORs in
    // SST_DEV_WAIT_EXPIRED when a bounded wait on a staged T row gave up (the
    // tile is then staged synchronously; results are unaffected), and
    // SST_DEV_COPY_LOST when the row copy had still not landed after a
    // second bounded wait
    unsigned *status;
    // test hook: CTA 0 does not issue its first row copy, so that wait expires
    int test_withhold;
    // one part of a signal split by frame ranges (sst_part_*): the pre-pass
    // takes only frames [frame_lo, frame_hi) (frame_hi = 0: every frame), and
    // the fused kernel's CTA b works on inverse tile tile0 + b
    int64_t frame_lo, frame_hi;
    int64_t tile0;
    // k_forward_alias: consecutive frames per chunk, whose samples are staged
    // in shared memory by one bulk copy (0: one frame per chunk)
    int fwd_chunk;
};
#define SST_DEV_WAIT_EXPIRED 0x1u
#define SST_DEV_COPY_LOST 0x2u

__host__ __device__ __forceinline__ bool in_zone(int l, int c, int hw) {
    return c >= 0 && (unsigned)(l - c + hw) <= (unsigned)(2 * hw);
}

__host__ __device__ __forceinline__ int64_t trow_of(const SstDev &d, int64_t m) {
    return d.trow_cap ? m % d.trow_cap : m;
}
__host__ __device__ __forceinline__ int64_t tslot_of(const SstDev &d, int64_t t) {
    return d.tile_cap ? t % d.tile_cap : t;
}

// Exact T sums.  A source's fixed-point value v = round(S^g 2^e) is kept
// below 2^SST_T_BITS / nb in magnitude (e from a bound on |S^g|), so a fine
// bin's sum of at most nb sources stays below 2^SST_T_BITS.  The sums are
// accumulated in shared memory as four arrays of 32-bit words (re lo, re hi,
// im lo, im hi), each tacc_stride(nbo) words long: v = hi 2^16 + lo with
// 0 <= lo < 2^16, so the lo sums of up to 2^16 sources stay below 2^32 and
// the hi sums below 2^31 -- exact, hence independent of the order of the
// (native 32-bit) atomic additions.
#define SST_T_BITS 45
__host__ __device__ __forceinline__ int tacc_stride(int nbo) { return (nbo + 3) & ~3; }
__host__ __device__ __forceinline__ size_t tacc_bytes(int nbo) { return 16 * (size_t)tacc_stride(nbo); }

// Per-call scalars produced on the device before the forward kernel runs
// (at the start of the workspace, or of the static scratch array).
struct SstScalars {
    float gamma2;   // threshold squared (relative plans)
    float maxv;     // max |S^g| over frames and band bins (relative plans)
    float s1, s2;   // fixed-point scale 2^e = s1 s2 for the exact T sums
    float r1, r2;   // its inverse 2^-e = r1 r2
    // one-pass relative threshold: sources above g_ub2 are kept at once, those
    // in (g_lb2, g_ub2] wait for the exact gamma, those at or below g_lb2 are dropped
    float g_lb2, g_ub2;
};

// One channel of a batch (sst_batch_*): its plan's device view (with the
// batch's own inverse tiling), its buffers and its slice of the workspace.
struct BatchChan {
    SstDev d;
    const float *x;
    float2 *T;
    float *xhat;
    SstScalars *sc;
    float *ola;        // overlap-add partials, d.ntiles x d.seg_len
    float frac2;       // relative threshold fraction squared
    float sum_abs_g;   // |S^g| <= max|x| sum|g| (absolute-threshold channels)
    int part0;         // first pre-pass partial of this channel
    int nparts;        // number of pre-pass partials of this channel
    int64_t poff;      // xhat holds samples from global index poff on (streams)
};

// A unit of batched work: channel `chan`, units [begin, end) -- quads of
// frames (pre-pass, relative channels), samples (pre-pass of absolute
// channels, finalize), frames (forward) or one inverse tile (begin).
struct BatchItem {
    int chan;
    int pad;
    int64_t begin, end;
};

}  // namespace sst
