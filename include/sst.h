/*
 * sst.h -- C ABI of libsst.so, the GB300 (sm_103a) implementation of the
 * downsampled STFT-based synchrosqueezing transform with selective
 * reassignment, frequency subdivision and the direct approximate inverse
 * (He & Cao, arXiv 2003.07065).
 *
 * Conventions shared by every call
 *  - Signals are float32.  Complex arrays (TFR, STFT) are interleaved float32
 *    pairs (re, im), row-major, one row per frame.
 *  - Frame m (0 <= m < F, F = ceil(n / hop)) is centred on sample m*hop; the
 *    signal is zero outside [0, n) (Sec. 2.1, Eq. 7-8).
 *  - Frequencies are in coarse DFT bins: bin k is k*fs/nfft Hz (Eq. 12).  The
 *    band [f_lo, f_hi] maps to bins k_lo = round(f_lo*nfft/fs),
 *    k_hi = round(f_hi*nfft/fs) (round half up), inclusive; N_r = k_hi - k_lo.
 *  - The squeezed TFR T has zN_r + 1 bins per frame: bin l sits at coarse
 *    frequency k_lo + l/z (Eq. 28-29).
 *  - Pointers named *_dev are device pointers; the caller allocates and owns
 *    them (e.g. through PyTorch), and they must stay valid until the work
 *    enqueued on `stream` has finished.  `stream` is a cudaStream_t passed as
 *    void*; NULL is the legacy default stream.  Calls enqueue work and return
 *    without synchronising unless stated otherwise.
 *  - `workspace_dev` is scratch device memory of at least the size returned
 *    by sst_plan_query (256-byte aligned).  Concurrent calls on different
 *    streams need distinct workspaces.
 *  - Every call validates its arguments before enqueueing anything and
 *    returns a status; it never throws or aborts.  A failed CUDA launch
 *    returns SST_ECUDA; asynchronous device faults surface on a later call
 *    or on sst_sync.  sst_last_error() gives a thread-local message for the
 *    last failure of the calling thread.
 *  - A plan is immutable after creation and may be shared by threads and
 *    streams.  It owns its device tables (window, twiddles, normaliser),
 *    allocated on the device that is current at creation; calls must be made
 *    with that device current.
 */
#ifndef SST_H
#define SST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SST_OK = 0,
    SST_EINVAL = 1,        /* invalid argument (message in sst_last_error) */
    SST_ENOMEM = 2,        /* host or device allocation failed */
    SST_ECUDA = 3,         /* a CUDA runtime call or launch failed */
    SST_EBUSY = 4,         /* no capacity (service admission) */
    SST_ETIMEOUT = 5,      /* a bounded device wait gave up */
    SST_EUNSUPPORTED = 6,  /* valid parameters this build does not handle */
    SST_EINTERNAL = 7      /* internal invariant violated */
} sst_status;

/* The longest window a plan takes (L = 2M + 1; any L up to it, longer than
 * nfft or not: the forward folds the window modulo nfft, exact by Eq. 8, and
 * the inverse evaluates Eq. 25 at every tap |n| <= M). */
#define SST_MAX_L 8193

/* flags */
#define SST_GAMMA_RELATIVE 0x1u  /* gamma is a fraction of max|V| over all frames and in-band bins */
/* Relative plans only: find max|V| in a separate full pass before the forward
 * transform (as the batch API does), instead of the default one-pass
 * threshold, which keeps every source clearly above the threshold, sets aside
 * those whose fate depends on the exact max|V| and settles them once the
 * forward pass has found it.  Both give the same kept set up to the rounding
 * of max|V| (the FP32 STFT of two different FFT packings); batch results are
 * bit-identical to single-plan results of plans with this flag. */
#define SST_TWO_PASS 0x2u

typedef struct sst_plan *sst_plan_t;

/* Parameters: the paper's own quantities (Sec. 2.1-2.4). */
typedef struct {
    int64_t n;          /* signal length N (samples), >= 1 */
    double fs;          /* sample rate in Hz (maps the band to bins, Eq. 12) */
    int32_t L;          /* odd window length L = 2M + 1, 1 < L <= SST_MAX_L; L > nfft is folded (Eq. 8) */
    double sigma;       /* Gaussian sigma in samples (Sec. 2.1), used when g == NULL */
    const double *g;    /* optional host window g[j], j = -M..M (L values), or NULL */
    const double *dg;   /* optional host derivative window g'[j] (Sec. 2.2); both or neither */
    int32_t hop;        /* time decimation H_t, 1 <= hop <= M */
    int32_t nfft;       /* DFT length N_f, a power of two in [64, 8192] (Eq. 9) */
    double f_lo, f_hi;  /* band of interest in Hz, 0 <= f_lo < f_hi <= fs/2 (Eq. 27) */
    int32_t z;          /* frequency subdivision factor, 1 <= z <= 16 (Eq. 28-29) */
    double gamma;       /* threshold on |V| (Eq. 13): absolute, or a fraction if SST_GAMMA_RELATIVE */
    uint32_t flags;
} sst_params;

/* Create a plan: validates the parameters, builds the window, twiddle and
 * inverse-normaliser tables in FP64 on the host, rounds them to FP32 and
 * uploads them (Sec. 2.1-2.3).  On success *out owns device memory until
 * sst_plan_destroy.  Errors: SST_EINVAL, SST_EUNSUPPORTED, SST_ENOMEM, SST_ECUDA. */
sst_status sst_plan_create(const sst_params *params, sst_plan_t *out);

/* Release a plan and its device tables.  NULL is ignored.  The caller must
 * make sure no enqueued work still uses the plan. */
void sst_plan_destroy(sst_plan_t plan);

/* Sizes of a plan: F frames, bins = zN_r + 1 TFR bins per frame, the band
 * k_lo..k_hi (inclusive, coarse bins) and the workspace the compute calls
 * need.  Any output pointer may be NULL. */
sst_status sst_plan_query(sst_plan_t plan, int64_t *frames, int32_t *bins,
                          int32_t *k_lo, int32_t *k_hi, size_t *workspace_bytes);

/* ---- Parameter guard (Sec. 4).  How far the frequency axis may be
 * downsampled before synchrosqueezing stops sharpening the TFR.  A Gaussian
 * window of standard deviation sigma_s seconds spreads a ridge over
 * sigma_f = 1 / (2 pi sigma_s) Hz (Eq. 35).  Coefficients still move to the
 * ridge while the coarse interval Delta f = fs / nfft = Hf fs / n (Eq. 12,
 * Hf = n / nfft) stays below 1.5 sigma_f (Eq. 37), i.e. Hf < 3 n / (4 pi
 * sigma_s fs) (Eq. 38), or, by the finite-difference model of Eq. 43-45,
 * below sqrt(2) sigma_f (Eq. 46), i.e. Hf < sqrt(2) sigma_f n / fs.
 * Subdivision (z) refines the output grid, not Delta f, so it does not
 * enter the bounds.  sigma_s = sigma / fs for the built-in window; for a
 * supplied window g it is taken from the second moment of g^2,
 * sigma^2 = 2 sum j^2 g[j]^2 / sum g[j]^2 (exact for a Gaussian). */
typedef struct {
    double sigma_s;          /* window standard deviation, seconds */
    double sigma_f_hz;       /* Eq. 35 */
    double hf;               /* Hf = n / nfft */
    double hf_max_eq38;      /* Eq. 38 bound on Hf */
    double hf_max_eq46;      /* Eq. 46 bound on Hf */
    double delta_f_hz;       /* coarse frequency interval fs / nfft (Eq. 12) */
    double delta_f_fine_hz;  /* output grid interval fs / (z nfft) (Eq. 28) */
    double delta_f_max_eq37_hz;  /* 1.5 sigma_f (Eq. 37) */
    double delta_f_max_eq46_hz;  /* sqrt(2) sigma_f (Eq. 46) */
    uint32_t flags;          /* SST_GUARD_*: the bounds Hf reaches or exceeds */
} sst_param_report;
#define SST_GUARD_EQ38 0x1u  /* Hf >= the Eq. 38 bound */
#define SST_GUARD_EQ46 0x2u  /* Hf >= the Eq. 46 bound */
/* Fills *out for a parameter set.  Host arithmetic only: no device is
 * needed or touched.  SST_EINVAL for parameters sst_plan_create rejects as
 * invalid (out untouched).  A plan beyond a bound is not an error: the flags
 * report it and the caller decides. */
sst_status sst_params_check(const sst_params *params, sst_param_report *out);
/* The same report for an existing plan. */
sst_status sst_plan_check(sst_plan_t plan, sst_param_report *out);

/* Forward SST (Sec. 2.2, 2.4): per frame, the packed Nf-point FFT of
 * x*g + i*x*g' gives S^g and S^g' (Eq. 9, split by Hermitian symmetry), the
 * IF estimate omega = k - (Nf/2pi) Im(S^g'/S^g) (Eq. 13), the threshold
 * |S^g| > gamma, and the in-band coefficients are summed into
 * T[m, l], l = floor(z (omega - k_lo) + 1/2) when 0 <= l <= zN_r (Eq. 27-29).
 * Sums are exact-then-rounded (deterministic, independent of thread order).
 *   x_dev   : n floats
 *   tfr_dev : F x bins complex (2*F*bins floats), fully overwritten
 * n must equal the plan's n. */
sst_status sst_forward(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev,
                       void *workspace_dev, void *stream);

/* Direct approximate inverse (Sec. 2.3, Eq. 25-26; zero padding and the
 * zNf-point inverse of Sec. 2.5): per frame
 *   r[m, j] = (2/Nf) Re sum_l w_l T[m,l] exp(i 2 pi (k_lo + l/z) j / Nf),
 *   j in [-M, M], w_l = 1/2 at the DC and Nyquist destinations, else 1;
 * then xhat[p] = sum_m g[p - m hop] r[m, p - m hop] / D[p] with
 * D[p] = g[0] sum_m g[p - m hop] (the exact discrete form of the 1/sqrt(2)
 * of Eq. 26).  Overlap-add order is fixed (deterministic).
 *   tfr_dev : F x bins complex;  xhat_dev : n floats, fully overwritten. */
sst_status sst_inverse(sst_plan_t plan, const float *tfr_dev, int64_t n, float *xhat_dev,
                       void *workspace_dev, void *stream);

/* Component recovery by time-frequency filtering (Sec. 2.3, last paragraph;
 * the zone M_q[m] of Eq. 15): sst_inverse of T with every coefficient
 * outside the zone set to zero.  Frame m's zone is the output bins l with
 * |l - ridge[m]| <= half_width, empty where ridge[m] < 0 (a ridge from
 * sst_ridge, or the caller's own IF track in output bins).
 *   ridge_dev  : F int32 on the device, 4-byte aligned, read only
 *   half_width : >= 0, in output bins (z per coarse bin)
 * T itself is not modified.  Errors: as sst_inverse, and SST_EINVAL for a
 * NULL or misaligned ridge or a negative half_width. */
sst_status sst_inverse_zone(sst_plan_t plan, const float *tfr_dev, int64_t n, const int32_t *ridge_dev,
                            int32_t half_width, float *xhat_dev, void *workspace_dev, void *stream);

/* Ridge of one component, one output bin per frame.  The paper extracts
 * ridges (Sec. 2.2 builds the Eq. 15 zone around them; Sec. 5 tracks IFs)
 * without stating a rule; this one is: E[m, l] = sum over |d| <= smooth,
 * 0 <= m + d < F, of |T[m + d, l]|^2 (FP32, d ascending), and ridge[m] is
 * the smallest l in [l_lo, l_hi] maximising E[m, l], or -1 when E[m, l] = 0
 * throughout.  Its frequency is (k_lo + l/z) fs/Nf.
 *   tfr_dev : frames x bins complex (row-major, 2*bins floats per frame),
 *             8-byte aligned
 *   0 <= l_lo <= l_hi < bins;  0 <= smooth <= SST_RIDGE_MAX_SMOOTH
 *   ridge_dev : frames int32, fully overwritten
 * No workspace; asynchronous on `stream`.  Errors: SST_EINVAL (pointers,
 * alignment, band or smooth out of range, before any CUDA call), SST_ECUDA. */
#define SST_RIDGE_MAX_SMOOTH 32
sst_status sst_ridge(const float *tfr_dev, int64_t frames, int32_t bins, int32_t l_lo, int32_t l_hi,
                     int32_t smooth, int32_t *ridge_dev, void *stream);

/* Renyi entropy of order alpha (Eq. 32; Sec. 3.2 uses alpha = 3) of the
 * distribution P = |T|^2 over a rows x cols grid (row stride ld complex
 * values): (1 / (1 - alpha)) log2 sum (P / sum P)^alpha + log2(cell), cell
 * being the area du dxi of a grid cell when the integrals are read as sums
 * over cells (1: the plain discrete form).  One pass over the data with a
 * running scale per thread (no overflow of P^alpha), partial sums combined
 * in FP64 in a fixed order (deterministic).
 *   alpha > 0, alpha != 1;  out_dev : one double on the device
 *   workspace_dev : sst_renyi_workspace_bytes() bytes, 256-byte aligned
 * Errors: SST_EINVAL (pointers, alignment, an empty grid, ld < cols, alpha,
 * cell; before any CUDA call), SST_ECUDA.  An all-zero grid gives NaN. */
size_t sst_renyi_workspace_bytes(void);
sst_status sst_renyi(const float *tfr_dev, int64_t rows, int32_t cols, int64_t ld, double alpha, double cell,
                     double *out_dev, void *workspace_dev, void *stream);

/* The whole path, forward (Sec. 2.2, 2.4) and direct inverse (Sec. 2.3).
 * With tfr_dev non-NULL: sst_forward followed by sst_inverse, T written to
 * tfr_dev and read back.  With tfr_dev NULL, T is not emitted and never
 * reaches global memory: the inverse of frame m needs only column m of T
 * (Eq. 25), so one kernel per tile of frames runs the forward of each pair
 * of frames into T rows in shared memory and inverts them from there
 * (Eq. 25-26).  With a relative threshold and the one-pass default, the
 * sources between the threshold's two bounds are left out of the rows and
 * recorded per tile; once the forward has found the exact max|S^g|, the
 * kept ones add their term of Eq. 25-26 to the reconstruction directly (in
 * the order of frame and source bin, so repeated calls give the same bits).
 * The kept sources are those of the same plan's call with a TFR output, and
 * the reconstructions differ by rounding only; should a tile's records
 * overflow, the call redoes itself with the two-pass kernels (behind a
 * device-side gate).  SST_TWO_PASS plans take max|S^g| from a pre-pass over
 * every frame and then carry the same bits as their call with a TFR output.
 * Plans whose fused kernel
 * would need more shared memory than the device offers per block (large Nf
 * with a wide band and subdivision) return SST_EUNSUPPORTED for a NULL
 * tfr_dev.  xhat_dev: n floats. */
sst_status sst_forward_inverse(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev,
                               float *xhat_dev, void *workspace_dev, void *stream);

/* End-to-end variant with host buffers: copies x_host (n floats, ideally
 * pinned) into x_dev, runs sst_forward_inverse (xhat_dev written as there)
 * and delivers the reconstruction into xhat_host: where xhat_host is
 * page-locked memory the device can address, the finalising kernel stores
 * it there directly, else it is copied from xhat_dev after the kernel.
 * Synchronises `stream` before returning. */
sst_status sst_forward_inverse_host(sst_plan_t plan, const float *x_host, int64_t n,
                                    float *xhat_host, float *x_dev, float *tfr_dev,
                                    float *xhat_dev, void *workspace_dev, void *stream);

/* In-band STFTs S^g and S^g' (Eq. 9, centre-referenced: phase factor
 * exp(i 2 pi k M / Nf) included), no threshold.  V_dev, Vd_dev: F x nb
 * complex with nb = k_hi - k_lo + 1.  For checking the transform. */
sst_status sst_stft(sst_plan_t plan, const float *x_dev, int64_t n, float *V_dev, float *Vd_dev,
                    void *workspace_dev, void *stream);

/* The reassignment map of sst_forward: omega_dev[m, k - k_lo] = the IF
 * estimate in coarse bins (Eq. 13, NaN where S^g = 0) and dest_dev = the
 * destination l, -1 below the threshold, -2 outside the grid.  F x nb each. */
sst_status sst_reassign_map(sst_plan_t plan, const float *x_dev, int64_t n, float *omega_dev,
                            int32_t *dest_dev, void *workspace_dev, void *stream);

/* ---- Second-order synchrosqueezing (the extension named in Sec. 6).  The
 * IF estimate of Eq. 13 is exact for a tone but biased off the ridge of a
 * chirp; the second-order estimate corrects it with the chirp rate, from the
 * STFTs with windows g, g', g'', t g and t g' (Eq. 8-9 conventions, t and
 * frequencies in samples and rad/sample):
 *   w~ = w + i S^{g'} / S^g,  q~ = i ((S^{g'})^2 - S^{g''} S^g) / (S^{tg} S^{g'} - S^{tg'} S^g),
 *   w2 = Re(w~ - q~ S^{tg} / S^g)   where |S^{tg} S^{g'} - S^{tg'} S^g| > 1e-3 |S^g|^2, else Re w~
 * (exact for linear chirps).  Threshold, grid and exact sums as sst_forward;
 * a relative threshold takes max|S^g| from a pre-pass over every frame.
 * Three packed FFTs per frame.  Needs the built-in Gaussian window
 * (SST_EUNSUPPORTED for a supplied one, or where the kernel's shared memory,
 * the frame buffer plus 16 bytes per fine bin plus 48 bytes per band bin,
 * exceeds the device's).  T from sst_forward2 inverts with sst_inverse. */
sst_status sst_forward2(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev, void *workspace_dev,
                        void *stream);
/* The map of sst_forward2: omega2_dev = the second-order IF in coarse bins
 * (NaN where S^g = 0), dest_dev as in sst_reassign_map.  F x nb each. */
sst_status sst_reassign_map2(sst_plan_t plan, const float *x_dev, int64_t n, float *omega2_dev,
                             int32_t *dest_dev, void *workspace_dev, void *stream);

/* max |S^g| over all frames and in-band bins (the base of a relative
 * threshold), written as one float to maxv_dev. */
sst_status sst_max_abs_v(sst_plan_t plan, const float *x_dev, int64_t n, float *maxv_dev,
                         void *workspace_dev, void *stream);

/* FP32 fused multiply-add throughput of the current device in TFLOP/s (2
 * FLOP per FMA), measured with eight independent fmaf chains per thread at
 * full occupancy: the denominator of an FP32 roofline.  Allocates 256 bytes,
 * launches three ~1 ms kernels on the stream and synchronises. */
sst_status sst_fp32_peak(double *tflops, void *stream);

/* The last sst_forward / sst_forward_inverse of a relative plan with the
 * one-pass threshold (the default): how many sources waited for the exact
 * threshold, how many fine bins they fell in (0 for a call without a TFR
 * output, which settles sources, not bins), and whether a record buffer
 * overflowed so that the two-pass kernels redid the call (then 1).  Reads
 * the control words the call left in `workspace` (synchronises the device).
 * Zeros for other plans. */
sst_status sst_threshold_stats(sst_plan_t plan, const void *workspace, int64_t *waiting, int64_t *bins,
                               int32_t *fell_back);

/* Status of the last sst_forward, sst_inverse, sst_inverse_zone or
 * sst_forward_inverse with a TFR output that used `workspace`.  The inverse
 * stages each pair of T rows in shared memory with one asynchronous bulk
 * copy, and the forward of pruning classes 1 and 2 each chunk of frames'
 * samples, each waited for with a bounded wait (about a second).  Should a
 * wait ever give up, the data are loaded with ordinary loads instead, so the
 * result is still correct, and this call reports SST_ETIMEOUT (with the
 * reason in sst_last_error).  Synchronises `stream`; SST_OK otherwise. */
sst_status sst_check(sst_plan_t plan, const void *workspace, void *stream);
/* Test hook of that path: in the next inverse of this plan one CTA does not
 * issue its first row copy, so its bounded waits run out (about two
 * seconds), it stages its tile synchronously and the next sst_check reports
 * SST_ETIMEOUT.  Nothing faults or hangs. */
sst_status sst_test_withhold_row_copy(sst_plan_t plan);
/* The same for the forward's staged samples: in the next sst_forward of
 * this plan one CTA does not issue its first sample copy (plans whose
 * forward stages its samples: pruning class 1 or 2). */
sst_status sst_test_withhold_sample_copy(sst_plan_t plan);

/* ---- One signal split by frame ranges, e.g. over several GPUs (one plan
 * per GPU, all with the same parameters).  Frames are independent (Sec. 2.1,
 * Eq. 7-9) and only the overlap-add of Eq. 26 couples neighbouring ones, so
 * part p of P takes a contiguous range of the plan's inverse tiles (tiles of
 * B frames) and reads only its frames' samples, a read-only halo of M
 * samples beyond them.  A relative threshold needs max |S^g| over every
 * frame: each part computes its own maximum (sst_part_prepass) and the
 * caller reduces them (a max over the parts, e.g. one all-reduce).  Each part
 * then runs the fused forward + inverse of its tiles (T stays on chip), which
 * leaves one overlap-add segment per tile in the workspace; the caller moves
 * the segments of tiles [need_begin, tile_begin) and [tile_end, need_end)
 * from the parts that computed them into the same places of this part's
 * workspace (sst_part_segments gives where), and sst_part_finalize divides
 * by D on the part's output samples.  The parts' outputs, concatenated,
 * carry the same bits as the unsplit sst_forward_inverse with a NULL tfr of
 * a SST_TWO_PASS plan (the parts' maximum is the exact one). */
typedef struct {
    int64_t tile_begin, tile_end;    /* the part's inverse tiles */
    int64_t frame_begin, frame_end;  /* its frames, [tile_begin B, min(tile_end B, F)) */
    int64_t x_begin, x_end;          /* the input samples it reads: its frames' windows, widened to
                                        whole groups of four frames (the pre-pass packs four) */
    int64_t out_begin, out_end;      /* the output samples it finalises */
    int64_t need_begin, need_end;    /* the tiles whose segments those samples need */
} sst_part;
/* The layout of part `part` of `parts` (host arithmetic; SST_EINVAL for a
 * part outside [0, parts)).  Parts tile the frames and the output samples. */
sst_status sst_part_layout(sst_plan_t plan, int32_t part, int32_t parts, sst_part *out);
/* Where the overlap-add segments live: tile t's seg_len floats start at byte
 * ola_offset + 4 seg_len t of the workspace; `tiles` tiles in all. */
sst_status sst_part_segments(sst_plan_t plan, size_t *ola_offset, int32_t *seg_len, int64_t *tiles);
/* The part's pre-pass maximum, one float written to r_dev: max |S^g|^2 over
 * its frames and the in-band bins (relative plans), or max |x| over its input
 * samples (absolute plans, the scale of the exact sums).  x_dev holds samples
 * [x_begin, x_end) of the signal. */
sst_status sst_part_prepass(sst_plan_t plan, const sst_part *part, const float *x_dev, float *r_dev,
                            void *workspace_dev, void *stream);
/* The part's forward + inverse, given r_dev = the maximum of every part's
 * pre-pass value: the overlap-add segments of tiles [tile_begin, tile_end)
 * in the workspace.  SST_EUNSUPPORTED where the plan's fused kernel does not
 * fit (see sst_forward_inverse). */
sst_status sst_part_forward_inverse(sst_plan_t plan, const sst_part *part, const float *x_dev, const float *r_dev,
                                    void *workspace_dev, void *stream);
/* x^ on the part's output samples into xhat_dev (out_end - out_begin floats),
 * from the segments of tiles [need_begin, need_end) in the workspace. */
sst_status sst_part_finalize(sst_plan_t plan, const sst_part *part, void *workspace_dev, float *xhat_dev,
                             void *stream);

/* Forward SST (as sst_forward) that allocates nothing and takes no
 * workspace.  The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc at the point where they run the transform, e.g. a
 * plug-in inside a host application whose device memory is entirely owned by
 * that application's own pool, or a latency-critical loop that must not hit
 * cudaMalloc's implicit device synchronisation.  (Creating the plan still
 * allocates its tables; do that at set-up time.)
 *   x_dev   : n floats; tfr_dev : F x bins complex, fully overwritten.
 * Scratch (the relative-threshold pre-pass's per-CTA maxima and gamma^2)
 * lives in one file-scope device array of SST_STATIC_SCRATCH_BYTES inside
 * libsst.so; every GPU that loads the library holds it until the process
 * exits.  Plans whose pre-pass needs more than the array holds are rejected
 * with SST_EUNSUPPORTED and a message giving both sizes.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.
 * The address is cached per device for the life of the process; it does not
 * survive cudaDeviceReset, so a process that resets a device must not call
 * this entry point on that device afterwards.
 * All calls share the one array and it keeps the last call's contents; every
 * element a call reads is written earlier in the same call, so nothing needs
 * clearing.  Calls whose work overlaps on the GPU (other streams, other
 * threads, other plans) race on the array: serialise them. */
#define SST_STATIC_SCRATCH_BYTES 65536
sst_status sst_forward_static(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev, void *stream);
/* Test hook: sst_forward_static treats the array as holding only `floats`
 * floats (0 restores its real size), so that its rejection of plans that
 * need more can be exercised. */
sst_status sst_test_static_capacity(size_t floats);

/* ---- Batched execution (many channels, uneven lengths, mixed parameters).
 * A batch groups the channels' work by DFT length and runs each group as one
 * persistent launch over a device table of work items (frame ranges,
 * inverse tiles); groups of the same phase run on parallel streams.  The
 * per-channel results are bit-identical to sst_forward_inverse on each item.
 * With SST_BATCH_GRAPH the whole launch sequence is captured into a CUDA
 * graph on the first sst_batch_run and replayed afterwards (re-captured if
 * the workspace or stream changes).  Plans and buffers must outlive the
 * batch. */
typedef struct {
    sst_plan_t plan;   /* the channel's plan */
    const float *x;    /* device, n floats */
    int64_t n;         /* must equal the plan's n */
    float *tfr;        /* device, F x bins complex */
    float *xhat;       /* device, n floats */
} sst_batch_item;
typedef struct sst_batch *sst_batch_t;
#define SST_BATCH_GRAPH 0x1u

/* Build the work tables (device memory owned by the batch).  Knobs come from
 * the tuning cache (in memory; also the file named by SST_TUNE_CACHE) when
 * a batch of the same shape class was tuned before, else defaults. */
sst_status sst_batch_create(const sst_batch_item *items, int32_t count, uint32_t flags, sst_batch_t *out);
/* Workspace bytes sst_batch_run needs (valid for every knob setting). */
sst_status sst_batch_workspace(sst_batch_t b, size_t *bytes);
/* Enqueue the whole batch (pre-pass, per-channel thresholds, forward,
 * inverse, finalize) on `stream`. */
sst_status sst_batch_run(sst_batch_t b, void *workspace_dev, void *stream);
/* Autotuner: times candidate work granularities and grid sizes on this
 * batch (runs it ~4 times per candidate; synchronises), keeps the fastest,
 * stores it in the tuning cache, and reports the untuned (default) and tuned
 * milliseconds per run. */
sst_status sst_batch_tune(sst_batch_t b, void *workspace_dev, void *stream, double *untuned_ms, double *tuned_ms);
/* Current knobs: frames per forward item, frame quads per pre-pass item, CTAs per SM multiplier. */
sst_status sst_batch_knobs(sst_batch_t b, int32_t *fwd_frames, int32_t *abs_quads, int32_t *grid_mul);
void sst_batch_destroy(sst_batch_t b);
/* One-shot: create, run, synchronise `stream`, destroy. */
sst_status sst_batch_submit(const sst_batch_item *items, int32_t count, void *workspace_dev, size_t workspace_bytes,
                            void *stream);
/* Workspace bytes sst_batch_submit needs for these items. */
sst_status sst_batch_workspace_for(const sst_batch_item *items, int32_t count, size_t *bytes);

/* ---- Streaming service (continuous batching of many live streams).
 * Streams push chunks of samples; each sst_service_tick moves every stream's
 * pending chunks to the device and runs, for all streams together, the
 * frames whose window has fully arrived, the inverse tiles (16 frames) whose
 * frames are all transformed, and the output samples no later frame touches.
 * Per-stream state (signal tail, TFR rows and overlap-add tiles not yet
 * consumed, cursors) stays on the device.  A stream's results do not depend
 * on its chunking or on the other streams; after sst_stream_close and the
 * ticks that flush it, they equal the whole-signal transform of the
 * concatenated chunks (absolute threshold).  Streams are admitted while their
 * device state fits the service's memory budget. */
typedef struct sst_service *sst_service_t;
sst_status sst_service_create(int32_t max_streams, size_t mem_budget_bytes, sst_service_t *out);
/* Open a stream.  params->n is ignored; the threshold must be absolute
 * (SST_EUNSUPPORTED otherwise: the whole-signal maximum is unknown while
 * streaming).  amp_bound >= max |x| of the stream fixes the exact-sum scale;
 * max_chunk bounds one push.  SST_EBUSY when no slot or budget is left. */
sst_status sst_stream_open(sst_service_t svc, const sst_params *params, float amp_bound, int64_t max_chunk,
                           int32_t *stream_id);
/* params->flags bit for sst_stream_open: deliver only the reconstruction;
 * the TFR columns stay on the device (ring) and are not copied to the host
 * (sst_stream_poll then returns no columns).  For services whose clients
 * want x-hat only: a TFR column is (zN_r + 1) complex values per hop, i.e.
 * 8 (zN_r + 1) / H bytes of host traffic per input sample. */
#define SST_STREAM_XHAT_ONLY 0x100u
/* Queue a host chunk (copied).  t_arrival: seconds on CLOCK_MONOTONIC (e.g.
 * Python time.monotonic()), or negative for "now"; latency = completion of
 * the tick that consumed the chunk minus t_arrival.  SST_EBUSY if more than
 * 8 max_chunk samples are queued. */
sst_status sst_stream_push(sst_service_t svc, int32_t stream_id, const float *host_chunk, int64_t n, double t_arrival);
/* End of data: later ticks flush the last frames (zero padding after the end). */
sst_status sst_stream_close(sst_service_t svc, int32_t stream_id);
/* Process everything ready on every stream; synchronous. */
sst_status sst_service_tick(sst_service_t svc);
/* Take finished output: up to max_cols TFR columns (bins complex each) and
 * up to max_samples reconstructed samples, with the index of the first of
 * each; *finished = 1 once a closed stream has delivered everything. */
sst_status sst_stream_poll(sst_service_t svc, int32_t stream_id, float *tfr_host, int64_t max_cols, int64_t *cols,
                           int64_t *first_col, float *xhat_host, int64_t max_samples, int64_t *samples,
                           int64_t *first_sample, int32_t *finished);
/* Free a stream's slot and device state. */
sst_status sst_stream_release(sst_service_t svc, int32_t stream_id);
/* Latency quantiles (seconds) over the chunks consumed so far; reset != 0 clears them. */
sst_status sst_service_latency(sst_service_t svc, double *p50, double *p99, int64_t *count, int32_t reset);
sst_status sst_service_memory(sst_service_t svc, size_t *used_bytes, size_t *budget_bytes);
void sst_service_destroy(sst_service_t svc);

/* Block until `stream` is idle; returns SST_ECUDA with the message of any
 * pending asynchronous error. */
sst_status sst_sync(void *stream);

/* Number of kernels this library has launched in this process (all
 * entry points, all threads). */
uint64_t sst_launch_count(void);

/* Tracing: every call that launches work (the transforms, the split-signal
 * parts, the batch and service calls, the post steps, plan creation, the
 * tensor form) opens an NVTX range named as the call for its duration, so a
 * timeline tool shows the calls above their kernels; without such a tool
 * attached NVTX does nothing.
 *
 * Per-kernel timing.  While enabled, each kernel launch of this library is
 * bracketed by two CUDA events recorded on the launch's own stream;
 * sst_profile_collect waits for them, adds the elapsed times per kernel kind
 * into ms[kind] and counts[kind] (arrays of SST_PROFILE_KINDS entries),
 * and clears the record.  Kinds: see sst_profile_kind_name. */
#define SST_PROFILE_KINDS 9
sst_status sst_profile_enable(int on);
sst_status sst_profile_collect(double *ms, uint64_t *counts);
const char *sst_profile_kind_name(int kind);

const char *sst_status_string(sst_status s);
const char *sst_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SST_H */
