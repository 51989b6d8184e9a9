/*
 * sst_tc.h -- C ABI of libsst_tc.so, the tensor-core band form of the
 * downsampled STFT-based synchrosqueezing transform (He & Cao, arXiv
 * 2003.07065): the in-band STFT pair of Eq. 8 as a dense contraction on the
 * tcgen05 tensor cores of one GB300, followed by the threshold, IF estimate
 * and reassignment of libsst.so.
 *
 * libsst_tc.so is a library of its own, linked against libsst.so, because
 * its contraction shares operand tiles between the CTAs of a cluster with
 * multicast TMA loads.  Those loads only ever read buffers the tensor plan
 * owns on the current device, and only single-GPU programs load this
 * library; nothing that runs on several GPUs at once builds or loads it.
 * The conventions of sst.h (status codes, device pointers, streams, error
 * messages through sst_last_error) apply unchanged.
 */
#ifndef SST_TC_H
#define SST_TC_H

#include "sst.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Tensor-core band form (precision study of the in-band bins).
 * Eq. 8 written as a direct sum over the L window taps for the band bins
 * k_lo..k_hi only (Sec. 2.4: only in-band bins feed the reassignment):
 *   [Re S^g, Im S^g, Re S^g', Im S^g'][m, k] = sum_j x[m H + j - M] B_c[j, k]
 * a [F x L] x [L x 4 nb] contraction on the tensor cores with FP32
 * accumulation, B built in FP64 from cos/sin(2 pi k (j - M) / Nf) times g and
 * g'.  Since no DFT of length Nf is taken, L > Nf needs no folding.  Forms:
 *   SST_FORM_BF16   : x and B rounded to BF16, one product;
 *   SST_FORM_BF16X3 : x = xh + xl, B = Bh + Bl in BF16; xh Bh + xh Bl + xl Bh;
 *   SST_FORM_TF32   : x and B as TF32 (10-bit mantissa), one product.
 * The threshold, IF estimate and reassignment (Eq. 13, 14) then run exactly as
 * in sst_forward, on the contraction's S^g and S^g'.
 * sst_tc_plan_create takes a plan made by sst_plan_create (it must outlive
 * the tensor plan) and allocates the operand and output buffers (about
 * (F + 4 nb) L elements plus an F x 4 nb FP32 product).  Errors: SST_EINVAL,
 * SST_EUNSUPPORTED (the driver gives no tensor-map encoder, or refuses the
 * operand layout), SST_ENOMEM, SST_ECUDA. */
#define SST_FORM_BF16 0
#define SST_FORM_BF16X3 1
#define SST_FORM_TF32 2
typedef struct sst_tc_plan *sst_tc_plan_t;
sst_status sst_tc_plan_create(sst_plan_t plan, int32_t form, sst_tc_plan_t *out);
void sst_tc_plan_destroy(sst_tc_plan_t tc);
/* hankel_view = 1 when the frames are read straight from the signal (rows H
 * samples apart), 0 when an explicit F x L copy is made; gemm_flops = the
 * multiply-adds x 2 of one contraction (all products of the form); cluster =
 * the CTAs that share each basis tile (sst_tc_plan_set_cluster). */
sst_status sst_tc_plan_query(sst_tc_plan_t tc, int32_t *hankel_view, int64_t *gemm_flops, int32_t *cluster);
/* How the contraction's CTAs share operands.  1, 2 or 4: CTAs per cluster;
 * each loads 1/cluster of the basis tile and multicasts it to the others
 * (M = 128 products per SM).  0: CTA pairs issuing one M = 256 product across
 * both SMs (tcgen05 cta_group::2), each SM loading its own rows and half of
 * the basis tile.  Results agree to the accumulation's rounding.
 * SST_EUNSUPPORTED if no such cluster fits. */
sst_status sst_tc_plan_set_cluster(sst_tc_plan_t tc, int32_t cluster);
/* Times the contraction on x_dev (n floats) with each cluster size that fits
 * (best of three after one untimed run, CUDA events on the stream), keeps the
 * fastest and returns it with its time in ms (either pointer may be NULL).
 * Synchronises the stream.  Errors as sst_tc_forward and sst_tc_check. */
sst_status sst_tc_plan_tune(sst_tc_plan_t tc, const float *x_dev, int64_t n, void *stream, int32_t *cluster,
                            float *ms);
/* As sst_forward / sst_stft / sst_reassign_map, through the contraction.
 * Layouts as there.  Enqueued on the stream without synchronising; the
 * contraction's waits are bounded, and one that gives up (about a second)
 * leaves its output undefined and is reported by the next sst_tc_check. */
sst_status sst_tc_forward(sst_tc_plan_t tc, const float *x_dev, int64_t n, float *tfr_dev, void *stream);
sst_status sst_tc_stft(sst_tc_plan_t tc, const float *x_dev, int64_t n, float *V_dev, float *Vd_dev, void *stream);
sst_status sst_tc_reassign_map(sst_tc_plan_t tc, const float *x_dev, int64_t n, float *omega_dev, int32_t *dest_dev,
                               void *stream);
/* The contraction alone (operand rounding and the product into the tensor
 * plan's own buffer), enqueued without synchronising: for timing. */
sst_status sst_tc_contract(sst_tc_plan_t tc, const float *x_dev, int64_t n, void *stream);
/* Synchronises the stream and returns SST_ETIMEOUT (and clears the record)
 * if any contraction of this tensor plan gave up a device wait since the
 * last check; SST_OK otherwise. */
sst_status sst_tc_check(sst_tc_plan_t tc, void *stream);
/* Test hook for the timeout path (cluster 1 only): in the next contraction
 * one CTA withholds its first operand load, so its bounded waits run out
 * after about a second each and the contraction returns early with its
 * output undefined; the next sst_tc_check reports SST_ETIMEOUT and the
 * context stays usable.  Nothing faults or hangs. */
sst_status sst_tc_plan_test_withhold(sst_tc_plan_t tc);

#ifdef __cplusplus
}
#endif
#endif /* SST_TC_H */
