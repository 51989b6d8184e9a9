// Kernels of the downsampled synchrosqueezing transform, templated on the
// DFT length NF.  One CTA of TPF threads works on one frame (forward) or one
// pair of frames (threshold pre-pass, inverse) at a time.  The frame gather
// (and, in the inverse, the spectrum build) is fused into the first FFT pass
// and the epilogue into the last one, so a frame makes three trips through
// shared memory for a 4096-point transform.
#pragma once
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sst_async.cuh"
#include "sst_dev.h"
#include "sst_fft.cuh"

namespace sst {

template <int NF> struct Cfg {
    static constexpr int TPF = (NF / 16 < 32) ? 32 : NF / 16;  // threads per CTA
    // float2 per frame buffer (the larger of the two layouts, rounded to 16 bytes)
    static constexpr int BUF = ((padded_len(NF) > dif_len<NF>() ? padded_len(NF) : dif_len<NF>()) + 1) & ~1;
    static constexpr int R1 = FftPlan<NF>::R1;                    // radix of the first pass
    static constexpr int PER1 = (NF / R1 + TPF - 1) / TPF;        // first-pass butterflies per thread
    static constexpr int NSL = NF / 16;                           // span of the last pass
    static constexpr int KMAX = (NF / 2 + 1 + TPF - 1) / TPF;     // band bins per thread
    static constexpr int NWARP = TPF / 32;
    // resident CTAs per SM the forward kernels are register-budgeted for
    static constexpr int MINB = (768 / TPF < 1) ? 1 : ((768 / TPF > 8) ? 8 : 768 / TPF);
};

// Pruning classes of the radix-16 first pass (STEP = NF / 16; a class is 0
// for any other first radix).  A band [k_lo, k_hi] of class 1 (k_hi < 3 STEP)
// and its mirror NF - k sit at positions j + r STEP with r in [0, 2] and
// [13, 15] only; class 2 (k_hi < 5 STEP): r in [0, 4] and [11, 15].  So the
// inverse's spectrum input and the forward's band output touch those r only.
// A forward of class c > 0 also has a window of L <= NF/2 + 1 taps, nonzero at
// r in [0, 4] and [12, 15] only.  Masks: bit r set = position r in use.
__host__ __device__ constexpr int band_class(int nf, int r1, int k_hi) {
    return r1 != 16 ? 0 : (k_hi < 3 * (nf / 16) ? 1 : (k_hi < 5 * (nf / 16) ? 2 : 0));
}
template <int NF> __host__ __device__ constexpr unsigned band_mask(int cls) {
    return (FftPlan<NF>::R1 != 16 || cls == 0) ? 0xffffu : (cls == 1 ? 0xE007u : 0xF81Fu);
}
template <int NF> __host__ __device__ constexpr unsigned window_mask(int cls) {
    return (FftPlan<NF>::R1 != 16 || cls == 0) ? 0xffffu : 0xF01Fu;
}
template <int NF> __host__ __device__ constexpr int cls_for(int cls) { return FftPlan<NF>::R1 == 16 ? cls : 0; }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// max over the CTA, result broadcast to every thread; uses red[NWARP]
template <int NWARP> __device__ __forceinline__ float block_max(float v, float *red, int tid) {
    v = warp_max(v);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float r = red[0];
#pragma unroll
    for (int w = 1; w < NWARP; ++w) r = fmaxf(r, red[w]);
    __syncthreads();
    return r;
}

// Windowed, folded frame sample at FFT position p (Eq. 8-9):
//   sum_{j = p mod NF, |j| <= M} x[c + j] * win[j]
// PAIR = false: win = (g, s g')  -> x (g + i s g');  s a power of two that
//               equalises the two halves' norms (undone exactly afterwards)
// PAIR = true : value (x[c1 + j] + i x[c2 + j]) g
template <int NF, bool PAIR>
__device__ __forceinline__ float2 frame_sample(const SstDev &d, const float *__restrict__ x, int p, int64_t c1,
                                               int64_t c2, bool has2) {
    float2 acc = make_float2(0.f, 0.f);
    const int jmin = p - NF * ((p + d.M) / NF);
    for (int j = jmin; j <= d.M; j += NF) {
        const float2 w = __ldg(&d.win[j + d.M]);
        const int64_t s1 = c1 + j;
        const float x1 = (s1 >= 0 && s1 < d.n) ? __ldg(&x[s1 - d.xoff]) : 0.f;
        if (!PAIR) {
            acc.x = fmaf(x1, w.x, acc.x);
            acc.y = fmaf(x1, w.y, acc.y);
        } else {
            const int64_t s2 = c2 + j;
            const float x2 = (has2 && s2 >= 0 && s2 < d.n) ? __ldg(&x[s2 - d.xoff]) : 0.f;
            acc.x = fmaf(x1, w.x, acc.x);
            acc.y = fmaf(x2, w.x, acc.y);
        }
    }
    return acc;
}

// First-pass inputs of one frame (or pair): u[b][r] = sample at FFT position
// j + r NF/R1, j = tid + b TPF.  Interior frames (window inside [0, n)) with
// L <= NF take a fast path: each position holds at most one tap, j = p or
// p - NF, read through 32-bit offsets from the frame centre.  Positions r
// whose bit in WMASK is clear hold no tap and are left unset.
template <int NF, bool PAIR, unsigned WMASK = 0xffffu>
__device__ __forceinline__ void gather_first(float2 (&u)[Cfg<NF>::PER1][Cfg<NF>::R1], const SstDev &d,
                                             const float *__restrict__ x, int64_t c1, int64_t c2, bool has2,
                                             int tid) {
    using C = Cfg<NF>;
    const bool in1 = c1 - d.M >= 0 && c1 + d.M < d.n;
    const bool in2 = !PAIR || (has2 && c2 - d.M >= 0 && c2 + d.M < d.n);
    if (in1 && in2 && d.L <= NF) {
        const float *x1 = x + (c1 - d.xoff);
        const float *x2 = x + ((PAIR ? c2 : c1) - d.xoff);
        const float2 *w = d.win + d.M;
#pragma unroll
        for (int b = 0; b < C::PER1; ++b) {
            const int j = tid + b * C::TPF;
#pragma unroll
            for (int r = 0; r < C::R1; ++r) {
                if (!((WMASK >> r) & 1u)) continue;
                const int p = j + r * (NF / C::R1);
                const bool lo = p <= d.M, hi = p >= NF - d.M;
                const int jj = lo ? p : p - NF;
                float2 val = make_float2(0.f, 0.f);
                if ((C::PER1 * C::TPF == NF / C::R1 || j < NF / C::R1) && (lo || hi)) {
                    const float2 wv = __ldg(&w[jj]);
                    const float a = __ldg(&x1[jj]);
                    if (!PAIR) val = make_float2(a * wv.x, a * wv.y);
                    else val = make_float2(a * wv.x, __ldg(&x2[jj]) * wv.x);
                }
                u[b][r] = val;
            }
        }
        return;
    }
#pragma unroll
    for (int b = 0; b < C::PER1; ++b) {
        const int j = tid + b * C::TPF;
#pragma unroll
        for (int r = 0; r < C::R1; ++r)
            if ((WMASK >> r) & 1u)
                u[b][r] = (C::PER1 * C::TPF == NF / C::R1 || j < NF / C::R1)
                              ? frame_sample<NF, PAIR>(d, x, j + r * (NF / C::R1), c1, c2, has2)
                              : make_float2(0.f, 0.f);
    }
}

// Forward FFT of frame(s) (c1, c2 are frame centres): gather fused into the
// first pass, outputs X[j + r NF/16] left in v (thread j = tid < NF/16).
// SYNC: end with a barrier, after which buf may be written.
template <int NF, bool PAIR, unsigned WMASK = 0xffffu, bool SYNC = true>
__device__ __forceinline__ void forward_fft(float2 *buf, const SstDev &d, const float *__restrict__ x, int64_t c1,
                                            int64_t c2, bool has2, int tid, float2 (&v)[16]) {
    using C = Cfg<NF>;
    float2 u[C::PER1][C::R1];
    gather_first<NF, PAIR, WMASK>(u, d, x, c1, c2, has2, tid);
    fft_in<NF, C::TPF, false, WMASK>(buf, u, d.tw, tid);
    __syncthreads();
    fft_mid<NF, C::TPF, false>(buf, d.tw, tid);
    fft_out<NF, C::TPF, false, SYNC>(buf, d.tw, tid, v);
}

// Scatter the last-pass outputs needed by the Hermitian split into buf:
// zc[k - k_lo] = X[k] and zm[k - k_lo] = X[(NF - k) mod NF] for k in the band.
// Only the positions r set in OMASK can hold a band bin.  Caller syncs
// afterwards.
template <int NF, unsigned OMASK = 0xffffu>
__device__ __forceinline__ void scatter_band(float2 *zc, float2 *zm, const SstDev &d, int tid, const float2 (&v)[16]) {
    constexpr int NS = NF / 16;
    if (Cfg<NF>::TPF == NS || tid < NS) {
        // k = q = tid + r NS lands at zc[kb0 + r NS] when 0 <= kb0 + r NS <= k_hi - k_lo,
        // its mirror NF - q at zm[km0 - r NS]: one unsigned compare per store
        const unsigned span = (unsigned)(d.k_hi - d.k_lo);
        const int kb0 = tid - d.k_lo, km0 = NF - tid - d.k_lo;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (!((OMASK >> r) & 1u)) continue;
            if ((unsigned)(kb0 + r * NS) <= span) zc[kb0 + r * NS] = v[r];
            if (r == 0 && tid == 0) {   // q = 0 is its own mirror
                if (d.k_lo == 0) zm[0] = v[0];
            } else if ((unsigned)(km0 - r * NS) <= span) {
                zm[km0 - r * NS] = v[r];
            }
        }
    }
}

// Store only the mirrors of the band: mz[k - k_lo] = X[(NF - k) mod NF] for k
// in the band (the zm half of scatter_band), for readers that take X[k]
// itself from the registers of thread k mod NF/16.  Caller syncs afterwards.
template <int NF, unsigned OMASK>
__device__ __forceinline__ void store_mirror(float2 *mz, const SstDev &d, int tid, const float2 (&v)[16]) {
    constexpr int NS = NF / 16;
    if (Cfg<NF>::TPF == NS || tid < NS) {
        const unsigned span = (unsigned)(d.k_hi - d.k_lo);
        const int km0 = NF - tid - d.k_lo;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (!((OMASK >> r) & 1u)) continue;
            if (r == 0 && tid == 0) {
                if (d.k_lo == 0) mz[0] = v[0];
            } else if ((unsigned)(km0 - r * NS) <= span) {
                mz[km0 - r * NS] = v[r];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Threshold pre-pass: max |S^g|^2 over in-band bins of every frame.  Two real
// frames share one complex FFT: Z = FFT((x_a + i x_b) g), S_a = (Z[k] +
// conj Z[-k]) / 2, S_b = (Z[k] - conj Z[-k]) / 2i.  Each thread carries two
// such FFTs at once (four frames per CTA iteration) to hide latency.  One
// partial max per CTA.
// ---------------------------------------------------------------------------
// CLS > 0 (a half-length window and a band of that pruning class): the first
// pass leaves out the inputs the window leaves zero and the scatter the
// positions no band bin occupies (the same values: only operations on exact
// zeros are left out)
template <int NF, int CLS = 0>
__device__ __forceinline__ float absmax_quad(const SstDev &d, const float *__restrict__ x, int64_t qq, float2 *buf,
                                             int tid, float best) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    constexpr int NB = 2;
    constexpr int BS = C::BUF;
    // FFT f (0, 1) packs frames a_f = 4 qq + 2 f and a_f + 1
    float2 u[NB][C::PER1][C::R1];
#pragma unroll
    for (int f = 0; f < NB; ++f) {
        const int64_t a = 4 * qq + 2 * f;
        const int64_t flo = d.frame_lo, fhi = d.frame_hi ? d.frame_hi : d.F;
        const bool hasa = a >= flo && a < fhi, hasb = a + 1 >= flo && a + 1 < fhi;
        const int64_t ca = hasa ? a * d.hop : -(int64_t)4 * NF - d.n;   // absent frame: all taps outside [0, n)
        gather_first<NF, true, window_mask<NF>(CLS)>(u[f], d, x, ca, (a + 1) * d.hop, hasb, tid);
    }
#pragma unroll
    for (int f = 0; f < NB; ++f) fft_first_from_regs<NF, TPF, false, window_mask<NF>(CLS)>(buf + f * BS, u[f], tid);
    __syncthreads();
    fft_middle_multi<NF, TPF, C::R1, false, NB, BS>(buf, d.tw, tid);
    float2 v[NB][16];
    fft_last_multi<NF, TPF, false, NB, BS>(buf, d.tw, tid, v);
#pragma unroll
    for (int f = 0; f < NB; ++f) scatter_band<NF, band_mask<NF>(CLS)>(buf + f * BS, buf + f * BS + d.nb, d, tid, v[f]);
    __syncthreads();
#pragma unroll
    for (int f = 0; f < NB; ++f) {
        const float2 *zc = buf + f * BS, *zm = zc + d.nb;
        for (int kk = tid; kk < d.nb; kk += TPF) {
            const float2 zk = zc[kk], zn = zm[kk];
            const float ar = 0.5f * (zk.x + zn.x), ai = 0.5f * (zk.y - zn.y);
            const float br = 0.5f * (zk.y + zn.y), bi = 0.5f * (zn.x - zk.x);
            best = fmaxf(best, fmaxf(ar * ar + ai * ai, br * br + bi * bi));
        }
    }
    __syncthreads();
    return best;
}

#define SST_ABSMAX_MINB ((512 / Cfg<NF>::TPF < 1) ? 1 : 512 / Cfg<NF>::TPF)

template <int NF, int CLS = 0>
__global__ void __launch_bounds__(Cfg<NF>::TPF, SST_ABSMAX_MINB)
k_absmax(SstDev d, const float *__restrict__ x, float *__restrict__ partial) {
    using C = Cfg<NF>;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    float *red = reinterpret_cast<float *>(buf + 2 * C::BUF);
    const int tid = threadIdx.x;
    if (d.gate && *d.gate == 0u) return;
    // quads of frames [frame_lo, frame_hi) (every frame when frame_hi = 0)
    const int64_t q_lo = d.frame_lo / 4, nquads = ((d.frame_hi ? d.frame_hi : d.F) + 3) / 4;
    const int64_t step = d.sample_stride > 1 ? d.sample_stride : 1;
    float best = 0.f;
    for (int64_t qq = q_lo + blockIdx.x * step; qq < nquads; qq += gridDim.x * step)
        best = absmax_quad<NF, CLS>(d, x, qq, buf, tid, best);
    best = block_max<C::NWARP>(best, red, tid);
    if (tid == 0) partial[blockIdx.x] = best;
}

// Reduce the pre-pass partial maxima into the call's scalars (see k_gamma in
// sst_capi.cu): threshold, max |S^g| and the fixed-point scale of the T sums.
// The call's scalars from the pre-pass maximum r.  Relative plans (from_x =
// 0): r = max |S^g|^2, gamma^2 = frac^2 r, maxv = sqrt(r).  Absolute plans
// (from_x = 1): r = max |x| and |S^g| <= max|x| sum|g|.  Either way the bound
// B on |S^g| (0.1% margin for the forward kernel's own rounding) gives the
// fixed-point scale 2^e, e = SST_T_BITS - ceil(log2 B) - ceil(log2 nb): a
// frame's at most nb terms then sum below 2^SST_T_BITS.
__device__ __forceinline__ SstScalars scalars_from_max(float r, float frac2, int from_x, float bound_mul,
                                                       int log2_nb) {
    SstScalars sc = {};
    float bound;
    if (!from_x) {
        const float mv = sqrtf(r);
        sc.gamma2 = frac2 * r;
        sc.maxv = mv;
        bound = mv * 1.001f;
    } else {
        bound = r * bound_mul;
    }
    int e = 0;
    if (bound > 0.f && bound < 3.0e38f) {
        int ex;
        frexpf(bound, &ex);  // bound < 2^ex
        e = SST_T_BITS - ex - log2_nb;
    }
    const int e1 = e / 2, e2 = e - e / 2;
    sc.s1 = ldexpf(1.f, e1);
    sc.s2 = ldexpf(1.f, e2);
    sc.r1 = ldexpf(1.f, -e1);
    sc.r2 = ldexpf(1.f, -e2);
    return sc;
}

__global__ void k_gamma(const float *__restrict__ partial, int count, float frac2, int from_x, float bound_mul,
                        int log2_nb, SstScalars *__restrict__ sc, float *__restrict__ maxv_out,
                        const unsigned *__restrict__ gate);

// Pre-pass of absolute-threshold plans: max |x| per CTA (bounds |S^g| by max|x| sum|g|).
__global__ void k_absx(const float *__restrict__ x, int64_t n, float *__restrict__ partial);

// ---------------------------------------------------------------------------
// Forward: per frame, packed FFT of x (g + i s g'), Hermitian split into S^g
// and S^g' for the band bins, IF estimate, threshold, destination, and the
// deterministic per-frame accumulation of T in shared memory.
//   MODE_T   : T rows (F x nbo complex)
//   MODE_TROW: as MODE_T, the frame's T row written to out0 itself (a
//              shared-memory row of the fused forward + inverse)
//   MODE_STFT: S^g, S^g' rows (F x nb complex each), no threshold
//   MODE_MAP : omega (F x nb float) and dest (F x nb int32)
// The T sum is exact: every contribution is scaled by the call's power of two
// 2^e (from the pre-pass bound on |S^g|, chosen so that any sum of a frame's
// terms stays below 2^62) and converted to int64 (exactly, for every term
// above 2^-39 of the bound); shared-memory 64-bit integer adds are order
// independent, so the rounded result does not depend on thread scheduling.
// ---------------------------------------------------------------------------
enum { MODE_T = 0, MODE_STFT = 1, MODE_MAP = 2, MODE_SPEC = 3, MODE_TROW = 4 };

// MODE_SPEC: per-frame shared-memory list of the sources that wait for the
// exact threshold (beyond it the call falls back to the two-pass path)
constexpr int SPEC_MCAP = 256;
struct SpecFrame {
    float4 item[SPEC_MCAP];    // (l as int bits, S^g re, S^g im, |S^g|^2)
    int binidx[SPEC_MCAP];     // the bin record of each listed source
};
// Records are taken from the global arrays in chunks of SPEC_CHUNK per CTA
// (one global atomic per chunk, not per frame); unused chunk tails are
// marked invalid (source bin -1, bin l -1).
constexpr unsigned SPEC_CHUNK = 256;
struct SpecCursor {
    unsigned src_cur, src_end, bin_cur, bin_end;
};
__device__ __forceinline__ void spec_drop_src(const SpecBuf &b, unsigned from, unsigned to) {
    for (unsigned i = from; i < to && i < (unsigned)b.cap_src; ++i) b.src[i].bin = -1;
}
__device__ __forceinline__ void spec_drop_bin(const SpecBuf &b, unsigned from, unsigned to) {
    for (unsigned i = from; i < to && i < (unsigned)b.cap_bin; ++i) b.bin[i].l = -1;
}
// k records from a chunk cursor (lane 0's registers); returns the first index
__device__ __forceinline__ unsigned spec_take(const SpecBuf &b, unsigned &cur, unsigned &end, unsigned k,
                                              unsigned *counter, bool src) {
    if (cur + k > end) {
        if (src) spec_drop_src(b, cur, end);
        else spec_drop_bin(b, cur, end);
        const unsigned take = max(SPEC_CHUNK, k);
        cur = atomicAdd(counter, take);
        end = cur + take;
    }
    const unsigned r = cur;
    cur += k;
    return r;
}
// Warp 0, after the frame's nm sources are listed: one bin record per
// distinct fine bin (with the exact sums of the sources already kept there,
// read before the accumulators are cleared), then one source record per
// listed source pointing at its bin's record.
__device__ __forceinline__ void spec_records(const SstDev &d, SpecFrame *sf, int nm, const uint32_t *acc,
                                             int64_t m, int lane, SpecCursor *cur) {
    const int n = min(nm, SPEC_MCAP);
    const int stride = tacc_stride(d.nbo);
    if (lane == 0 && nm > SPEC_MCAP) d.spec.ctl[3] = 1u;
    for (int c = 0; c < n; c += 32) {
        const int i = c + lane;
        const int l = i < n ? __float_as_int(sf->item[i].x) : -1;
        int first = i;   // the earliest listed source with the same bin
        if (i < n)
            for (int j = 0; j < i; ++j)
                if (__float_as_int(sf->item[j].x) == l) { first = j; break; }
        const bool lead = i < n && first == i;
        const unsigned lm = __ballot_sync(0xffffffffu, lead);
        unsigned base = 0;
        if (lane == 0 && lm) {
            base = spec_take(d.spec, cur->bin_cur, cur->bin_end, (unsigned)__popc(lm), &d.spec.ctl[2], false);
            atomicAdd(&d.spec.ctl[6], (unsigned)__popc(lm));   // statistics (no wait)
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lead) {
            const unsigned b = base + (unsigned)__popc(lm & ((1u << lane) - 1u));
            if (b < (unsigned)d.spec.cap_bin) {
                SpecBin r;
                r.m = m;
                r.l = l;
                r.w[0] = acc[l];
                r.w[1] = acc[stride + l];
                r.w[2] = acc[2 * stride + l];
                r.w[3] = acc[3 * stride + l];
                r.pad = 0;
                d.spec.bin[b] = r;
                sf->binidx[i] = (int)b;
            } else {
                d.spec.ctl[3] = 1u;
                sf->binidx[i] = -1;
            }
        }
        __syncwarp();
        if (i < n && !lead) sf->binidx[i] = sf->binidx[first];
        __syncwarp();
    }
    unsigned sbase = 0;
    if (lane == 0 && n) {
        sbase = spec_take(d.spec, cur->src_cur, cur->src_end, (unsigned)n, &d.spec.ctl[1], true);
        atomicAdd(&d.spec.ctl[5], (unsigned)n);
    }
    sbase = __shfl_sync(0xffffffffu, sbase, 0);
    for (int i = lane; i < n; i += 32) {
        const unsigned g = sbase + (unsigned)i;
        if (g < (unsigned)d.spec.cap_src) {
            const float4 it = sf->item[i];
            SpecSrc r;
            r.bin = sf->binidx[i];
            r.vr = it.y;
            r.vi = it.z;
            r.mag2 = it.w;
            d.spec.src[g] = r;
        } else {
            d.spec.ctl[3] = 1u;
        }
    }
}
// bytes of the band's mirror values (forward kernels of class > 0)
__host__ __device__ constexpr size_t mirror_bytes(int nb) { return (8 * (size_t)nb + 15) & ~(size_t)15; }
// bytes of MODE_SPEC shared state (one SpecFrame, whatever the row length)
__host__ __device__ __forceinline__ size_t spec_smem_bytes(int /*nbo*/) {
    return sizeof(SpecFrame);
}
// whether it fits in a frame buffer of buf float2 after the 2 nb band values
__host__ __device__ __forceinline__ bool spec_in_frame(int nb, int nbo, int buf) {
    return ((16 * (size_t)nb + 15) & ~(size_t)15) + spec_smem_bytes(nbo) <= 8 * (size_t)buf;
}

struct FwdScale {
    float gamma2;   // threshold squared (MODE_SPEC: the lower one, g_lb2)
    float s1, s2;   // fixed-point scale 2^e = s1 s2
    float r1, r2;   // 2^-e = r1 r2
    float g_ub2;    // MODE_SPEC: above this a source is kept without waiting
};

__device__ __forceinline__ FwdScale fwd_scale(const SstDev &d, const SstScalars *__restrict__ sc, bool need_t) {
    FwdScale f;
    f.gamma2 = d.relative ? sc->gamma2 : d.gamma2_abs;
    f.s1 = f.s2 = f.r1 = f.r2 = 1.f;
    f.g_ub2 = 0.f;
    if (need_t) { f.s1 = sc->s1; f.s2 = sc->s2; f.r1 = sc->r1; f.r2 = sc->r2; }
    return f;
}

// The fixed-point value a = round(x) (round half to even, |x| < 2^45) split
// as a = hi 2^16 + lo, 0 <= lo < 2^16, without a 64-bit conversion (several
// times slower here): below 2^23 through a 32-bit one; above, x is already an
// integer and x - floor(x / 2^16) 2^16 is exact.
__device__ __forceinline__ void tacc_split(float x, uint32_t &lo, uint32_t &hi) {
    if (fabsf(x) < 8388608.f) {
        const int a = __float2int_rn(x);
        lo = (uint32_t)a & 0xffffu;
        hi = (uint32_t)(a >> 16);
    } else {
        const float hf = floorf(x * (1.f / 65536.f));
        lo = (uint32_t)(int)fmaf(-hf, 65536.f, x);
        hi = (uint32_t)(int)hf;
    }
}

// Adds a source (V scaled by 2^e) to fine bin l of the T accumulators.
__device__ __forceinline__ void tacc_add(uint32_t *__restrict__ acc, int stride, int l, float2 V, const FwdScale &fs) {
    uint32_t alo, ahi, blo, bhi;
    tacc_split((V.x * fs.s1) * fs.s2, alo, ahi);
    tacc_split((V.y * fs.s1) * fs.s2, blo, bhi);
    atomicAdd(&acc[l], alo);
    atomicAdd(&acc[stride + l], ahi);
    atomicAdd(&acc[2 * stride + l], blo);
    atomicAdd(&acc[3 * stride + l], bhi);
}

// The exact sum v = hi 2^16 + lo (|v| < 2^45) rounded once to float.  v is
// split as h 2^21 + r with |h| < 2^24 and 0 <= r < 2^21, both exact in float,
// and one fused multiply-add rounds h 2^21 + r: the correctly rounded value,
// as a 64-bit integer conversion would give, from 32-bit conversions only
// (the 64-bit one is several times slower here).
__device__ __forceinline__ float tacc_value(uint32_t lo, uint32_t hi, const FwdScale &fs) {
    const long long v = ((long long)(int32_t)hi << 16) + (long long)lo;
    const int h = (int)(v >> 21);
    const int r = (int)(v & 0x1fffff);
    return (fmaf((float)h, 2097152.f, (float)r) * fs.r1) * fs.r2;
}

// Reads fine bins 4 q .. 4 q + 3 (those below nbo) into Trow and (CLEAR)
// clears them.
template <bool CLEAR = true>
__device__ __forceinline__ void tacc_take4(uint32_t *__restrict__ acc, int stride, int q, int nbo,
                                           float2 *__restrict__ Trow, const FwdScale &fs) {
    uint4 *a4 = reinterpret_cast<uint4 *>(acc);
    const int s4 = stride >> 2;
    const uint4 rl = a4[q], rh = a4[s4 + q], il = a4[2 * s4 + q], ih = a4[3 * s4 + q];
    if (CLEAR) {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        a4[q] = z;
        a4[s4 + q] = z;
        a4[2 * s4 + q] = z;
        a4[3 * s4 + q] = z;
    }
    const float2 t0 = make_float2(tacc_value(rl.x, rh.x, fs), tacc_value(il.x, ih.x, fs));
    const float2 t1 = make_float2(tacc_value(rl.y, rh.y, fs), tacc_value(il.y, ih.y, fs));
    const float2 t2 = make_float2(tacc_value(rl.z, rh.z, fs), tacc_value(il.z, ih.z, fs));
    const float2 t3 = make_float2(tacc_value(rl.w, rh.w, fs), tacc_value(il.w, ih.w, fs));
    const int l = 4 * q;
    if (l + 3 < nbo && (reinterpret_cast<uintptr_t>(Trow + l) & 15) == 0) {
        reinterpret_cast<float4 *>(Trow + l)[0] = make_float4(t0.x, t0.y, t1.x, t1.y);
        reinterpret_cast<float4 *>(Trow + l)[1] = make_float4(t2.x, t2.y, t3.x, t3.y);
    } else {
        Trow[l] = t0;
        if (l + 1 < nbo) Trow[l + 1] = t1;
        if (l + 2 < nbo) Trow[l + 2] = t2;
        if (l + 3 < nbo) Trow[l + 3] = t3;
    }
}

// Band bin kk (k = k_lo + kk) of frame m from X[k] = zk and X[NF - k] = zn:
// the Hermitian split, then by MODE the STFT pair, the map entry, or the
// reassignment of the source into the T accumulators (MODE_SPEC: sources
// between the threshold bounds are listed in sf instead, *nmarg counting them).
template <int MODE>
__device__ __forceinline__ void frame_bin(const SstDev &d, const FwdScale &fs, float2 *__restrict__ out0,
                                          void *__restrict__ out1, int64_t m, int kk, float2 zk, float2 zn,
                                          uint32_t *acc, SpecFrame *sf, int *nmarg, float *vmax) {
    const int k = d.k_lo + kk;
    const float2 V = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
    const float2 Vd = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
    const size_t o = (size_t)m * d.nb + kk;
    if (MODE == MODE_STFT) {
        out0[o] = V;
        reinterpret_cast<float2 *>(out1)[o] = make_float2(Vd.x * d.dscale, Vd.y * d.dscale);
        return;
    }
    const float mag2 = V.x * V.x + V.y * V.y;
    // reassignment offset in bins: -(Nf / 2 pi) Im(S^g' / S^g)   (Eq. 13, 36).
    // The quotient by the fast reciprocal is within 2 ulp for a divisor in
    // [2^-126, 2^126]; the (rare) others take the IEEE division.
    const float num = Vd.y * V.x - Vd.x * V.y;
    float quo;
    if (mag2 >= 0x1p-126f && mag2 <= 0x1p126f) quo = __fdividef(num, mag2);
    else quo = num / mag2;
    const float delta = -d.c_if * quo;
    int l = -1;
    if (mag2 > fs.gamma2) {
        const float f = floorf(fmaf((float)d.z, delta, 0.5f));
        l = -2;
        if (f > -1073741824.f && f < 1073741824.f) {
            const int lc = d.z * (k - d.k_lo) + (int)f;
            if (lc >= 0 && lc < d.nbo) l = lc;
        }
    }
    if (MODE == MODE_MAP) {
        reinterpret_cast<float *>(out0)[o] = (mag2 > 0.f) ? (float)k + delta : __int_as_float(0x7fc00000);
        reinterpret_cast<int32_t *>(out1)[o] = l;
        return;
    }
    if (MODE == MODE_SPEC) {
        *vmax = fmaxf(*vmax, mag2);
        if (l >= 0 && !(mag2 > fs.g_ub2)) {
            // kept only if |S^g| exceeds the exact threshold: list it, flag its bin
            const int i = atomicAdd(nmarg, 1);
            if (i < SPEC_MCAP) sf->item[i] = make_float4(__int_as_float(l), V.x, V.y, mag2);
            return;
        }
    }
    if (MODE == MODE_TROW && d.fused_count) {
        // the one-pass threshold of the path without a TFR output: a source
        // between the bounds is left out of the row and recorded for the
        // settling pass, which adds its share of the reconstruction if the
        // exact threshold keeps it (*nmarg: the tile's record count)
        *vmax = fmaxf(*vmax, mag2);
        if (l >= 0 && !(mag2 > fs.g_ub2)) {
            const int i = atomicAdd(nmarg, 1);
            if (i < d.fused_cap) {
                SpecBin r;
                r.m = m;
                r.l = l;
                r.w[0] = __float_as_uint(V.x);
                r.w[1] = __float_as_uint(V.y);
                r.w[2] = __float_as_uint(mag2);
                r.w[3] = (uint32_t)kk;
                r.pad = 0;
                d.fused_rec[(size_t)(m / d.B) * d.fused_cap + i] = r;
            } else {
                atomicOr(&d.spec.ctl[3], 1u);   // the gated two-pass kernels redo the call
            }
            return;
        }
    }
    if (l >= 0) tacc_add(acc, tacc_stride(d.nbo), l, V, fs);
}

// One frame m of the forward transform.  The T accumulators (tacc_stride(nbo) words x 4) must be
// zero on entry and are zero again on return (MODE_T, MODE_SPEC).  MODE_SPEC
// also needs sf and nmarg (both set up here for every frame; nmarg outside
// the frame buffer) and the CTA's record cursor, and folds max |S^g|^2 into
// *vmax.  CLS: pruning class (see band_class); for CLS > 0 the band values
// X[k] stay in the registers of the thread that computed them and only the
// mirrors X[NF - k] pass through mz (nb float2 outside the frame buffer), so
// the last FFT pass needs no barrier of its own.
template <int NF, int MODE, int CLS = 0>
__device__ __forceinline__ void forward_frame(const SstDev &d, const float *__restrict__ x, const FwdScale &fs,
                                              float2 *__restrict__ out0, void *__restrict__ out1, int64_t m,
                                              float2 *buf, uint32_t *acc, int tid, SpecFrame *sf = nullptr,
                                              int *nmarg = nullptr, float *vmax = nullptr,
                                              SpecCursor *cur = nullptr, float2 *mz = nullptr) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    constexpr int NS = NF / 16;
    constexpr bool REG = CLS > 0;
    constexpr unsigned OMASK = band_mask<NF>(CLS);
    float2 v[16];
    forward_fft<NF, false, window_mask<NF>(CLS), !REG>(buf, d, x, m * d.hop, 0, false, tid, v);
    float2 *zc = buf, *zm = buf + d.nb;
    if constexpr (REG) store_mirror<NF, OMASK>(mz, d, tid, v);
    else scatter_band<NF, OMASK>(zc, zm, d, tid, v);
    if (MODE == MODE_SPEC && tid == 0) *nmarg = 0;
    __syncthreads();

    if constexpr (REG) {
        if (TPF == NS || tid < NS) {
            const unsigned span = (unsigned)(d.k_hi - d.k_lo);
            const int kb0 = tid - d.k_lo;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                if (!((OMASK >> r) & 1u)) continue;
                const int kk = kb0 + r * NS;
                if ((unsigned)kk <= span) frame_bin<MODE>(d, fs, out0, out1, m, kk, v[r], mz[kk], acc, sf, nmarg, vmax);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < C::KMAX; ++i) {
            const int kk = tid + i * TPF;
            if (kk < d.nb) frame_bin<MODE>(d, fs, out0, out1, m, kk, zc[kk], zm[kk], acc, sf, nmarg, vmax);
        }
    }
    // all band reads and atomics done before the T row is read and the next
    // frame's first pass overwrites buf
    __syncthreads();
    if (MODE != MODE_T && MODE != MODE_SPEC && MODE != MODE_TROW) return;
    float2 *Trow = MODE == MODE_TROW ? out0 : out0 + (size_t)trow_of(d, m) * d.nbo;
    const int stride = tacc_stride(d.nbo);
    if (MODE == MODE_SPEC) {
        const int nm = *nmarg;
        if (nm > 0) {   // (block-uniform)
            if (tid < 32) spec_records(d, sf, nm, acc, m, tid, cur);
            __syncthreads();   // records read the sums before they are cleared, and sf before the next FFT
        }
    }
    for (int q = tid; 4 * q < d.nbo; q += TPF) tacc_take4(acc, stride, q, d.nbo, Trow, fs);
    // the zeroing above is ordered before the next frame's atomics by the
    // __syncthreads inside the next frame's FFT
}

template <int NF, int MODE, int CLS = 0>
__global__ void __launch_bounds__(Cfg<NF>::TPF, Cfg<NF>::MINB)
k_forward(SstDev d, const float *__restrict__ x, const SstScalars *__restrict__ sc,
          float2 *__restrict__ out0, void *__restrict__ out1) {
    using C = Cfg<NF>;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    // after the frame buffer (BUF float2 = BUF x 8 bytes) and 128 bytes of slack:
    // the T accumulators
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem4) + 2 * C::BUF + 32;
    const int tid = threadIdx.x;
    if (d.gate && *d.gate == 0u) return;
    FwdScale fs = fwd_scale(d, sc, MODE == MODE_T || MODE == MODE_SPEC);
    if (MODE == MODE_SPEC) {
        fs.gamma2 = sc->g_lb2;
        fs.g_ub2 = sc->g_ub2;
    }
    const int stride = tacc_stride(d.nbo);
    // CLS > 0: the band's mirror values after the accumulators
    float2 *mz = reinterpret_cast<float2 *>(acc + 4 * stride);
    // MODE_SPEC state: the source counter in the frame buffer's slack; the
    // list in the frame buffer after the band values when it fits there (no
    // extra shared memory, so no loss of occupancy), else after the
    // accumulators (and the mirrors)
    int *nmarg = reinterpret_cast<int *>(buf + C::BUF);
    const size_t band_bytes = (16 * (size_t)d.nb + 15) & ~(size_t)15;
    SpecFrame *sf = (spec_in_frame(d.nb, d.nbo, C::BUF))
                        ? reinterpret_cast<SpecFrame *>(reinterpret_cast<char *>(buf) + band_bytes)
                        : reinterpret_cast<SpecFrame *>(reinterpret_cast<char *>(mz) + (CLS > 0 ? mirror_bytes(d.nb) : 0));
    if (MODE == MODE_T || MODE == MODE_SPEC)
        for (int i = tid; i < 4 * stride; i += C::TPF) acc[i] = 0u;
    float vmax = 0.f;
    SpecCursor cur = {0u, 0u, 0u, 0u};
    // (the first __syncthreads in forward_frame orders this before any atomic)
    for (int64_t m = blockIdx.x; m < d.F; m += gridDim.x)
        forward_frame<NF, MODE, CLS>(d, x, fs, out0, out1, m, buf, acc, tid, sf, nmarg, &vmax, &cur, mz);
    if (MODE == MODE_SPEC) {
        vmax = warp_max(vmax);
        if ((tid & 31) == 0 && vmax > 0.f) atomicMax(&d.spec.ctl[0], __float_as_uint(vmax));
        if (tid == 0) {
            spec_drop_src(d.spec, cur.src_cur, cur.src_end);
            spec_drop_bin(d.spec, cur.bin_cur, cur.bin_end);
        }
    }
}

// ---------------------------------------------------------------------------
// Second-order synchrosqueezing (the extension Sec. 6 names): the IF estimate
// of a frame's bin corrected for the chirp rate.  From the STFTs with windows
// g, g', g'', t g and t g' (in samples; Eq. 8-9 conventions), with w the
// bin's frequency in rad/sample:
//   complex IF    w~ = w + i V^{g'} / V                 (Re: Eq. 13)
//   chirp rate    q~ = i ((V^{g'})^2 - V^{g''} V) / (V^{tg} V^{g'} - V^{tg'} V)
//   second order  w2 = Re(w~ - q~ V^{tg} / V),  where |V^{tg} V^{g'} - V^{tg'} V| > 1e-3 |V|^2
//                 (else the chirp rate is ill-conditioned: w2 = Re w~)
// The five STFTs come from three packed FFTs per frame: x (g + i s1 g'),
// x (s2 g'' + i s3 t g) and x s4 t g' (each s a power of two equalising
// norms, undone exactly).  Reassignment, threshold and the exact sums are
// those of the first-order forward.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cdiv_scaled(float2 a, float2 b) {
    // a / b with both scaled by 1 / max(|b.x|, |b.y|) (no overflow of |b|^2)
    const float m = fmaxf(fabsf(b.x), fabsf(b.y));
    const float s = 1.0f / m;
    const float2 bs = make_float2(b.x * s, b.y * s), as = make_float2(a.x * s, a.y * s);
    const float den = bs.x * bs.x + bs.y * bs.y;
    return make_float2((as.x * bs.x + as.y * bs.y) / den, (as.y * bs.x - as.x * bs.y) / den);
}

// Band bin kk of frame m from the three packed FFTs' band values (zc, zm
// layout of scatter_band for each): MODE_MAP writes the second-order IF (bins)
// and the destination, MODE_T adds the source to the T accumulators.
template <int MODE>
__device__ __forceinline__ void frame_bin_so(const SstDev &d, const FwdScale &fs, float2 *__restrict__ out0,
                                             void *__restrict__ out1, int64_t m, int kk, const float2 *A,
                                             const float2 *B, const float2 *C, uint32_t *acc) {
    const int k = d.k_lo + kk, nb = d.nb;
    float2 zk = A[kk], zn = A[nb + kk];
    const float2 V = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
    const float2 Vd = make_float2(0.5f * (zk.y + zn.y) * d.dscale, 0.5f * (zn.x - zk.x) * d.dscale);
    zk = B[kk];
    zn = B[nb + kk];
    const float2 V2 = make_float2(0.5f * (zk.x + zn.x) * d.r2, 0.5f * (zk.y - zn.y) * d.r2);
    const float2 Vt = make_float2(0.5f * (zk.y + zn.y) * d.r3, 0.5f * (zn.x - zk.x) * d.r3);
    zk = C[kk];
    zn = C[nb + kk];
    const float2 Vtd = make_float2(0.5f * (zk.x + zn.x) * d.r4, 0.5f * (zk.y - zn.y) * d.r4);
    const float mag2 = V.x * V.x + V.y * V.y;
    float delta = __int_as_float(0x7fc00000);
    if (mag2 > 0.f) {
        const float c = d.c_so;                     // Nf / (2 pi): rad/sample -> bins
        const float2 ratio = cdiv_scaled(Vd, V);    // V^{g'} / V
        delta = -c * ratio.y;                       // Re(i ratio) in bins: the first-order offset
        const float2 den = csub(cmul(Vt, Vd), cmul(Vtd, V));
        if (hypotf(den.x, den.y) > 1e-3f * mag2) {
            const float2 num = csub(cmul(Vd, Vd), cmul(V2, V));
            const float2 qq = cdiv_scaled(num, den);            // q~ / i
            const float2 q = make_float2(-qq.y, qq.x);          // q~
            const float2 corr = cmul(q, cdiv_scaled(Vt, V));    // q~ V^{tg} / V
            delta -= c * corr.x;
        }
    }
    int l = -1;
    if (mag2 > fs.gamma2) {
        const float f = floorf(fmaf((float)d.z, delta, 0.5f));
        l = -2;
        if (f > -1073741824.f && f < 1073741824.f) {
            const int lc = d.z * (k - d.k_lo) + (int)f;
            if (lc >= 0 && lc < d.nbo) l = lc;
        }
    }
    if (MODE == MODE_MAP) {
        const size_t o = (size_t)m * d.nb + kk;
        reinterpret_cast<float *>(out0)[o] = (mag2 > 0.f) ? (float)k + delta : __int_as_float(0x7fc00000);
        reinterpret_cast<int32_t *>(out1)[o] = l;
        return;
    }
    if (l >= 0) tacc_add(acc, tacc_stride(d.nbo), l, V, fs);
}

// bytes of k_forward_so's shared memory: the frame buffer (+ slack), the T
// accumulators, and the band values of the three FFTs (2 nb float2 each)
__host__ __device__ inline size_t forward_so_smem_bytes(size_t smem_frame, int nb, int nbo) {
    return smem_frame + tacc_bytes(nbo) + 6 * 8 * (size_t)nb;
}

#define SST_SO_MINB ((512 / Cfg<NF>::TPF < 1) ? 1 : 512 / Cfg<NF>::TPF)

template <int NF, int MODE>
__global__ void __launch_bounds__(Cfg<NF>::TPF, SST_SO_MINB)
k_forward_so(SstDev d, const float *__restrict__ x, const SstScalars *__restrict__ sc, float2 *__restrict__ out0,
             void *__restrict__ out1) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem4) + 2 * C::BUF + 32;
    const int stride = tacc_stride(d.nbo);
    float2 *band = reinterpret_cast<float2 *>(acc + 4 * stride);
    float2 *bA = band, *bB = band + 2 * d.nb, *bC = band + 4 * d.nb;
    const int tid = threadIdx.x;
    const FwdScale fs = fwd_scale(d, sc, MODE == MODE_T);
    for (int i = tid; i < 4 * stride; i += TPF) acc[i] = 0u;
    SstDev d2 = d, d3 = d;
    d2.win = d.win2;
    d3.win = d.win3;
    for (int64_t m = blockIdx.x; m < d.F; m += gridDim.x) {
        float2 v[16];
        forward_fft<NF, false>(buf, d, x, m * d.hop, 0, false, tid, v);     // ends with a barrier
        scatter_band<NF>(bA, bA + d.nb, d, tid, v);
        forward_fft<NF, false>(buf, d2, x, m * d.hop, 0, false, tid, v);
        scatter_band<NF>(bB, bB + d.nb, d, tid, v);
        forward_fft<NF, false>(buf, d3, x, m * d.hop, 0, false, tid, v);
        scatter_band<NF>(bC, bC + d.nb, d, tid, v);
        __syncthreads();
        for (int kk = tid; kk < d.nb; kk += TPF) frame_bin_so<MODE>(d, fs, out0, out1, m, kk, bA, bB, bC, acc);
        __syncthreads();   // the bins read and the atomics done before the read-out and the next frame
        if (MODE == MODE_T) {
            float2 *Trow = out0 + (size_t)trow_of(d, m) * d.nbo;
            for (int q = tid; 4 * q < d.nbo; q += TPF) tacc_take4(acc, stride, q, d.nbo, Trow, fs);
        }
    }
}

// ---------------------------------------------------------------------------
// The forward of a pruning class > 0 with the T accumulators in the frame
// buffer.  Such a forward keeps the band values in registers after the last
// FFT pass and the mirrors outside the frame buffer, so the buffer is free
// from the end of the last pass until the next frame's first pass: the
// accumulators (cleared there each frame) take its place, which more than
// halves the shared memory of a CTA and lets four CTAs (32 warps) share an
// SM instead of three.  Same arithmetic as k_forward; two more barriers per
// frame.  A CTA takes chunks of d.fwd_chunk consecutive frames; the chunk's
// samples ((chunk - 1) hop + L of them, zero outside [0, n)) are staged in
// shared memory by one bulk copy where the range is 16-byte aligned and
// inside the signal, else by plain loads, and every frame of the chunk
// gathers its windowed taps from there.  Shared memory: the frame buffer
// (BUF float2; the accumulators alias its start), 128 bytes of slack (the
// MODE_SPEC counter), the band mirrors, the MODE_SPEC list, the chunk's
// samples and the copy's mbarrier.
// ---------------------------------------------------------------------------
#define SST_FWDA_MINB ((1024 / Cfg<NF>::TPF < 1) ? 1 : ((1024 / Cfg<NF>::TPF > 8) ? 8 : 1024 / Cfg<NF>::TPF))

// floats of the staged samples of a chunk (rounded up so the copy's length
// is a multiple of 16 bytes, plus that rounding's slack)
__host__ __device__ constexpr int fwd_seg_floats(int chunk, int hop, int L) {
    return (((chunk - 1) * hop + L + 3) & ~3) + 4;
}
__host__ __device__ constexpr size_t forward_alias_smem_bytes(int nf_buf, int nb, bool spec, int seg_floats) {
    return 8 * (size_t)nf_buf + 128 + mirror_bytes(nb) + (spec ? ((sizeof(SpecFrame) + 15) & ~(size_t)15) : 0) +
           4 * (size_t)seg_floats + 16;
}
// whether the accumulators of nbo fine bins fit in a frame buffer of nf_buf float2
__host__ __device__ inline bool tacc_fits_frame(int nbo, int nf_buf) { return tacc_bytes(nbo) <= 8 * (size_t)nf_buf; }

// First-pass inputs of one frame from staged samples: seg[off + j] is the
// sample at the frame's centre + j (zero outside the signal), taps j with
// |j| <= M, at most one per position (L <= NF).  The same products as
// gather_first's interior path.
template <int NF, unsigned WMASK>
__device__ __forceinline__ void gather_staged(float2 (&u)[Cfg<NF>::PER1][Cfg<NF>::R1], const SstDev &d,
                                              const float *seg, int off, int tid) {
    using C = Cfg<NF>;
    const float2 *w = d.win + d.M;
    const float *xs = seg + off;
#pragma unroll
    for (int b = 0; b < C::PER1; ++b) {
        const int j = tid + b * C::TPF;
#pragma unroll
        for (int r = 0; r < C::R1; ++r) {
            if (!((WMASK >> r) & 1u)) continue;
            const int p = j + r * (NF / C::R1);
            const bool lo = p <= d.M, hi = p >= NF - d.M;
            const int jj = lo ? p : p - NF;
            float2 val = make_float2(0.f, 0.f);
            if ((C::PER1 * C::TPF == NF / C::R1 || j < NF / C::R1) && (lo || hi)) {
                const float2 wv = __ldg(&w[jj]);
                const float a = xs[jj];
                val = make_float2(a * wv.x, a * wv.y);
            }
            u[b][r] = val;
        }
    }
}

template <int NF, int MODE, int CLS>
__device__ __forceinline__ void forward_frame_alias(const SstDev &d, const float *seg, int off, const FwdScale &fs,
                                                    float2 *__restrict__ out0, int64_t m, float2 *buf, int tid,
                                                    SpecFrame *sf, int *nmarg, float *vmax, SpecCursor *cur,
                                                    float2 *mz) {
    static_assert(CLS > 0, "the band values must stay in registers");
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    constexpr int NS = NF / 16;
    constexpr unsigned OMASK = band_mask<NF>(CLS), WMASK = window_mask<NF>(CLS);
    uint32_t *acc = reinterpret_cast<uint32_t *>(buf);
    const int stride = tacc_stride(d.nbo);
    float2 v[16];
    {
        float2 u[C::PER1][C::R1];
        gather_staged<NF, WMASK>(u, d, seg, off, tid);
        fft_in<NF, TPF, false, WMASK>(buf, u, d.tw, tid);
    }
    __syncthreads();
    fft_mid<NF, TPF, false>(buf, d.tw, tid);
    fft_out<NF, TPF, false, true>(buf, d.tw, tid, v);   // ends with a barrier
    store_mirror<NF, OMASK>(mz, d, tid, v);
    uint4 *a4 = reinterpret_cast<uint4 *>(acc);
    for (int i = tid; i < stride; i += TPF) a4[i] = make_uint4(0u, 0u, 0u, 0u);   // 4 stride words
    if (MODE == MODE_SPEC && tid == 0) *nmarg = 0;
    __syncthreads();
    if (TPF == NS || tid < NS) {
        const unsigned span = (unsigned)(d.k_hi - d.k_lo);
        const int kb0 = tid - d.k_lo;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (!((OMASK >> r) & 1u)) continue;
            const int kk = kb0 + r * NS;
            if ((unsigned)kk <= span) frame_bin<MODE>(d, fs, out0, nullptr, m, kk, v[r], mz[kk], acc, sf, nmarg, vmax);
        }
    }
    __syncthreads();
    float2 *Trow = out0 + (size_t)trow_of(d, m) * d.nbo;
    if (MODE == MODE_SPEC) {
        const int nm = *nmarg;
        if (nm > 0) {   // (block-uniform)
            if (tid < 32) spec_records(d, sf, nm, acc, m, tid, cur);
            __syncthreads();
        }
    }
    // (the accumulators live in the frame buffer, which the next frame's FFT
    // overwrites and which is cleared again after it: no clearing here)
    for (int q = tid; 4 * q < d.nbo; q += TPF) tacc_take4<false>(acc, stride, q, d.nbo, Trow, fs);
    // the read-out (and this frame's reads of the staged samples) done before
    // the next frame's first pass overwrites the buffer, or the next chunk's copy the samples
    __syncthreads();
}

template <int NF, int MODE, int CLS>
__global__ void __launch_bounds__(Cfg<NF>::TPF, SST_FWDA_MINB)
k_forward_alias(SstDev d, const float *__restrict__ x, const SstScalars *__restrict__ sc,
                float2 *__restrict__ out0, void *__restrict__ out1) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    int *nmarg = reinterpret_cast<int *>(buf + C::BUF);
    float2 *mz = reinterpret_cast<float2 *>(reinterpret_cast<char *>(smem4) + 8 * (size_t)C::BUF + 128);
    SpecFrame *sf = reinterpret_cast<SpecFrame *>(reinterpret_cast<char *>(mz) + mirror_bytes(d.nb));
    const int chunk = d.fwd_chunk > 0 ? d.fwd_chunk : 1;
    const int seg_floats = fwd_seg_floats(chunk, d.hop, d.L);
    float *seg = reinterpret_cast<float *>(reinterpret_cast<char *>(sf) +
                                           (MODE == MODE_SPEC ? ((sizeof(SpecFrame) + 15) & ~(size_t)15) : 0));
    uint64_t *bar = reinterpret_cast<uint64_t *>(seg + seg_floats);
    const int tid = threadIdx.x;
    if (d.gate && *d.gate == 0u) return;
    FwdScale fs = fwd_scale(d, sc, true);
    if (MODE == MODE_SPEC) {
        fs.gamma2 = sc->g_lb2;
        fs.g_ub2 = sc->g_ub2;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    float vmax = 0.f;
    SpecCursor cur = {0u, 0u, 0u, 0u};
    uint32_t phase = 0;
    bool bulk = true;   // cleared for the rest of the launch should a copy's wait ever expire
    bool withheld = false;  // (test hook: CTA 0 withholds only its first copy)
    const int64_t nchunks = (d.F + chunk - 1) / chunk;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t m0 = c * chunk;
        const int64_t m1 = m0 + chunk < d.F ? m0 + chunk : d.F;
        const int64_t s0 = m0 * d.hop - d.M;
        const int len = (int)((m1 - 1 - m0) * d.hop) + d.L;
        const int len4 = (len + 3) & ~3;
        const float *src = x + (s0 - d.xoff);
        // staging: one bulk copy where it may run (16-byte aligned, inside the
        // signal), with a bounded wait; else, or should the wait expire, loads
        bool staged = false;
        if (bulk && s0 >= 0 && s0 + len4 <= d.n && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            int ok = 1;
            if (tid == 0) {
                mbar_expect_tx(bar, 4u * (uint32_t)len4);
                // (test hook: CTA 0 does not issue its first copy, so its waits expire)
                if (!(d.test_withhold && blockIdx.x == 0 && !withheld)) bulk_g2s(seg, src, 4u * (uint32_t)len4, bar);
                ok = mbar_wait(bar, phase) ? 1 : 0;
                if (!ok) {
                    const bool landed = mbar_wait(bar, phase);
                    if (d.status) atomicOr(d.status, SST_DEV_WAIT_EXPIRED | (landed ? 0u : SST_DEV_COPY_LOST));
                }
            }
            phase ^= 1u;
            withheld = true;
            staged = __syncthreads_and(ok) != 0;
            bulk = staged;
        }
        if (!staged) {
            // (a late copy would write these same values)
            for (int i = tid; i < len; i += TPF) {
                const int64_t sp = s0 + i;
                seg[i] = (sp >= 0 && sp < d.n) ? __ldg(&x[sp - d.xoff]) : 0.f;
            }
            __syncthreads();
        }
        for (int64_t m = m0; m < m1; ++m)
            forward_frame_alias<NF, MODE, CLS>(d, seg, (int)((m - m0) * d.hop) + d.M, fs, out0, m, buf, tid, sf,
                                               nmarg, &vmax, &cur, mz);
    }
    if (MODE == MODE_SPEC) {
        vmax = warp_max(vmax);
        if ((tid & 31) == 0 && vmax > 0.f) atomicMax(&d.spec.ctl[0], __float_as_uint(vmax));
        if (tid == 0) {
            spec_drop_src(d.spec, cur.src_cur, cur.src_end);
            spec_drop_bin(d.spec, cur.bin_cur, cur.bin_end);
        }
    }
}

// ---------------------------------------------------------------------------
// Inverse, one CTA per tile of B consecutive frames (B even), frames taken in
// pairs (a, b = a + 1).  r_a + i r_b comes out of z complex inverse FFTs of
// length NF: sub-grid s (fine bins l = z q + s) is placed at coarse bin
// k_lo + q together with the Hermitian image of sub-grid (z - s) mod z, and
// the result at tap j is multiplied by exp(i 2 pi s j / (z NF)) (Eq. 25, with
// the zNf-point zero-padded inverse of Sec. 2.5 split into its z interleaved
// sub-grids).  The sub-grids are taken in descending order and their
// results summed by Horner's rule in omega = exp(i 2 pi j / (z NF)), one
// complex multiply-add per tap and sub-grid.  The pair's two T rows are
// staged in shared memory; the spectrum build is fused into the first FFT
// pass and the tap accumulation into the last, whose thread j holds the
// outputs q = j + r NF/16.  NARROW (L <= NF/2 + 1) keeps the 9 accumulators of
// r in [0, 4] and [12, 15]; otherwise (L <= NF + 1) all 16 plus the tap -NF/2
// (which shares q = NF/2 with +NF/2); a longer window has no accumulators
// (inverse_long_sub).  The windowed frames are overlap-added into a
// shared-memory segment in ascending frame order, written to the partial
// buffer, and k_finalize sums overlapping segments in tile order and applies
// 1 / D[p] (Eq. 26).
// ---------------------------------------------------------------------------
template <bool NARROW> struct InvTaps {
    static constexpr int NACC = NARROW ? 9 : 17;
    // r of accumulator i (i = 16 is the extra tap -NF/2 at r = 8)
    __host__ __device__ static constexpr int r_of(int i) { return NARROW ? (i <= 4 ? i : i + 7) : (i < 16 ? i : 8); }
};

// The last-pass taps of thread tid: n_i = q or q - NF (q = tid + r NF/16),
// INT_MIN where outside the window, and (NARROW) omega_i = exp(2 pi i n_i /
// (z NF)), the sub-grid twiddle of sub-grid 1, whose powers give the others.
template <int NF, bool NARROW>
__device__ __forceinline__ void inverse_taps(const SstDev &d, int tid, int (&tap)[InvTaps<NARROW>::NACC],
                                             float2 (&om)[InvTaps<NARROW>::NACC]) {
    using TP = InvTaps<NARROW>;
    constexpr int NS = NF / 16;
    const bool live = (Cfg<NF>::TPF == NS) || tid < NS;
    const float2 b1 = (NARROW && d.z > 1 && live) ? __ldg(&d.twb[NS + tid]) : make_float2(1.f, 0.f);
#pragma unroll
    for (int i = 0; i < TP::NACC; ++i) {
        const int r = TP::r_of(i);
        const int q = tid + r * NS;
        int n;
        if (i == 16) n = -NF / 2;
        else n = (r < 8 || (r == 8 && tid == 0)) ? q : q - NF;
        const bool ok = live && n >= -d.M && n <= d.M && !(i == 16 && tid != 0);
        tap[i] = ok ? n : INT_MIN;
        om[i] = make_float2(1.f, 0.f);
        if (NARROW && ok && d.z > 1) om[i] = cmul(b1, __ldg(&d.twc[(2 + (n < 0)) * 16 + r]));
    }
}

// First FFT pass of sub-grid s of a pair of rows (a, b), with the spectrum
// built in registers: Y_s[k] = X_a,s[k] + conj X_a,sb[-k-dl]
// + i (X_b,s[k] + conj X_b,sb[-k-dl]), sb = (z - s) mod z, dl = (s > 0).
// Element q of sub-grid s of row a is Ta[q qstride] (Tam for sub-grid sb;
// Tb, Tbm for row b).  Input k = j + r NF/R1 reads q = k - k_lo and, for the
// image, qm = ((NF - k - dl) mod NF) - k_lo = (NF - dl - j - k_lo) - r NF/R1,
// except at k = 0 with dl = 0 (qm = -k_lo).  The coarse DC and Nyquist bins
// (k = 0 and NF/2 of sub-grid 0, i.e. j = 0 with r = 0 or R1/2) are their own
// images: both terms land on the same input, which takes the weight 1/2.
// The band is a small part of the spectrum, so most r hold nothing for a
// whole warp: those iterations are skipped on a warp vote.  No barrier inside.
template <int NF, int CLS>
__device__ __forceinline__ void inverse_first_pass(const SstDev &d, const float2 *Ta, const float2 *Tam,
                                                   const float2 *Tb, const float2 *Tbm, int qstride, int s,
                                                   float2 *buf, int tid) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    constexpr int STEP = NF / C::R1;
    const int nq = d.k_hi - d.k_lo + 1;
    const int sb = (s == 0) ? 0 : d.z - s;
    const int dl = (s == 0) ? 0 : 1;
    const int nqs = (s == 0) ? nq : nq - 1;     // sub-grid s holds q in [0, nqs)
    const int nqb = (sb == 0) ? nq : nq - 1;
    float2 u[C::PER1][C::R1];
#pragma unroll
    for (int bb = 0; bb < C::PER1; ++bb) {
        const int j = tid + bb * TPF;
        const bool jok = C::PER1 * TPF == NF / C::R1 || j < NF / C::R1;
        const int q0 = j - d.k_lo;
        const int qm0 = NF - dl - j - d.k_lo;
#pragma unroll
        for (int r = 0; r < C::R1; ++r) {
            if (!((band_mask<NF>(CLS) >> r) & 1u)) continue;
            float2 y = make_float2(0.f, 0.f);
            const int q = q0 + r * STEP;
            const int qm = (r == 0 && j == 0 && dl == 0) ? -d.k_lo : qm0 - r * STEP;
            const bool hd = jok && (unsigned)q < (unsigned)nqs;
            const bool hm = jok && (unsigned)qm < (unsigned)nqb;
            if (__any_sync(0xffffffffu, hd || hm)) {
                if (hd) {
                    const float2 xa = Ta[q * qstride], xb = Tb[q * qstride];
                    y.x += xa.x - xb.y;
                    y.y += xa.y + xb.x;
                }
                if (hm) {
                    const float2 xa = Tam[qm * qstride], xb = Tbm[qm * qstride];
                    // conj(xa) + i conj(xb)
                    y.x += xa.x + xb.y;
                    y.y += -xa.y + xb.x;
                }
                if ((r == 0 || r == C::R1 / 2) && s == 0 && j == 0) y = cscale(y, 0.5f);
            }
            u[bb][r] = y;
        }
    }
    fft_in<NF, TPF, true, band_mask<NF>(CLS)>(buf, u, d.tw, tid);
}

// shared memory of the inverse: frame buffer, the pair's rows by sub-grid, overlap-add segment
__host__ __device__ inline size_t inverse_smem_bytes(size_t smem_frame, int z, int nq, int seg_len) {
    return smem_frame + 16 * (size_t)z * (size_t)nq + 4 * (size_t)seg_len;
}

// Overlap-add of one frame's taps (the real part: frame a of the pair; the
// imaginary part: frame b) into the segment at offset o, each weighted by
// g[n_i] / NF (the inverse DFT's 1 / NF, a power of two, so exact, applied
// once per tap instead of to every spectrum input).
template <int NF, bool NARROW, bool IMAG>
__device__ __forceinline__ void inverse_ola(const SstDev &d, float *seg, int o,
                                            const int (&tap)[InvTaps<NARROW>::NACC],
                                            const float2 (&racc)[InvTaps<NARROW>::NACC]) {
    const float cnorm = 1.0f / (float)NF;
#pragma unroll
    for (int i = 0; i < InvTaps<NARROW>::NACC; ++i)
        if (tap[i] != INT_MIN) seg[o + tap[i]] += (__ldg(&d.g[tap[i] + d.M]) * cnorm) * (IMAG ? racc[i].y : racc[i].x);
}

// The same with the weights read once for both frames of the pair, all loads
// before the first store: for kernels whose plan descriptor lives in shared
// memory (batches), where each store to the segment would otherwise make the
// compiler read the window pointer and M again before the next tap's load.
template <int NF, bool NARROW>
__device__ __forceinline__ void inverse_weights(const SstDev &d, const int (&tap)[InvTaps<NARROW>::NACC],
                                                float (&gw)[InvTaps<NARROW>::NACC]) {
    const float cnorm = 1.0f / (float)NF;
    const float *g = d.g + d.M;
#pragma unroll
    for (int i = 0; i < InvTaps<NARROW>::NACC; ++i) gw[i] = tap[i] != INT_MIN ? __ldg(&g[tap[i]]) * cnorm : 0.f;
}
template <bool NARROW, bool IMAG>
__device__ __forceinline__ void inverse_ola_w(float *seg, int o, const int (&tap)[InvTaps<NARROW>::NACC],
                                              const float (&gw)[InvTaps<NARROW>::NACC],
                                              const float2 (&racc)[InvTaps<NARROW>::NACC]) {
#pragma unroll
    for (int i = 0; i < InvTaps<NARROW>::NACC; ++i)
        if (tap[i] != INT_MIN) seg[o + tap[i]] += gw[i] * (IMAG ? racc[i].y : racc[i].x);
}

// Tap accumulation of sub-grid s, taken in descending order (Horner's rule
// in omega): racc = sum_s omega^s v_s, i.e. every tap gets the sub-grid
// twiddle exp(i 2 pi s n / (z NF)) of Eq. 25's zNf-point inverse.  The 9
// taps of a half-length window keep omega in registers (om); the 17 of a
// wider one form it again from the tables at each sub-grid (holding 17 more
// complex values would spill).
template <int NF, bool NARROW>
__device__ __forceinline__ void inverse_accumulate(const SstDev &d, float2 (&racc)[InvTaps<NARROW>::NACC],
                                                   const float2 (&v)[16], const float2 (&om)[InvTaps<NARROW>::NACC],
                                                   const int (&tap)[InvTaps<NARROW>::NACC], int tid, bool first) {
    using TP = InvTaps<NARROW>;
    if constexpr (NARROW) {
#pragma unroll
        for (int i = 0; i < TP::NACC; ++i) {
            const float2 x = v[TP::r_of(i)];
            if (first) {
                racc[i] = x;
            } else {
                const float2 a = racc[i], w = om[i];
                racc[i] = make_float2(fmaf(a.x, w.x, fmaf(-a.y, w.y, x.x)), fmaf(a.x, w.y, fmaf(a.y, w.x, x.y)));
            }
        }
    } else {
        if (first) {
#pragma unroll
            for (int i = 0; i < TP::NACC; ++i) racc[i] = v[TP::r_of(i)];
            return;
        }
        const float2 b1 = __ldg(&d.twb[NF / 16 + tid]);
#pragma unroll
        for (int i = 0; i < TP::NACC; ++i) {
            const float2 x = v[TP::r_of(i)];
            const float2 w = (i == 16) ? __ldg(&d.twn[1]) : cmul(b1, __ldg(&d.twc[(2 + (tap[i] < 0)) * 16 + TP::r_of(i)]));
            const float2 a = racc[i];
            racc[i] = make_float2(fmaf(a.x, w.x, fmaf(-a.y, w.y, x.x)), fmaf(a.x, w.y, fmaf(a.y, w.x, x.y)));
        }
    }
}

// The inverse and fused kernels' class for a window longer than NF + 1: no
// pruning, and the taps go through inverse_long_sub (NARROW false).
constexpr int CLS_LONG = -1;

// Sub-grid s of a pair for a window longer than NF + 1 (Eq. 25 at every tap
// n in [-M, M]).  Tap n reads output q = n mod NF of each sub-grid, so thread
// tid's 16 outputs q = tid + r NF/16 serve the taps n = q + w NF inside the
// window, any number of them per q; a Horner accumulator per tap would take
// about 16 L / NF complex registers, so instead each sub-grid's term
// (g[n] / NF) exp(i 2 pi s n / (z NF)) v_s[q] goes straight into the
// segment: its real part at frame a's taps, then, after a barrier, its
// imaginary part at frame b's.  Every sample's sum runs over the sub-grids
// in descending order, frame a before frame b, whatever the thread count.
// All threads take the barrier; callers order the next frame-a stores
// behind this call's frame-b stores with a barrier of their own.
template <int NF>
__device__ __forceinline__ void inverse_long_sub(const SstDev &d, float *seg, int oa, bool hasb,
                                                 const float2 (&v)[16], int s, int tid, bool live) {
    constexpr int NS = NF / 16;
    const int G = d.z * NF;
    const float cnorm = 1.0f / (float)NF;
    for (int f = 0; f < 2; ++f) {
        if (f == 1) __syncthreads();
        if (!live || (f == 1 && !hasb)) continue;
        const int o = oa + f * d.hop;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int q = tid + r * NS;
            for (int n = q - NF * ((q + d.M) / NF); n <= d.M; n += NF) {
                float2 c = v[r];
                if (s > 0) {
                    int k = (s * n) % G;
                    if (k < 0) k += G;
                    c = cmul(__ldg(&d.twf[k]), c);
                }
                seg[o + n] += (__ldg(&d.g[n + d.M]) * cnorm) * (f ? c.y : c.x);
            }
        }
    }
}

// One inverse tile; smem4 is the kernel's dynamic shared memory.  Ends with a
// barrier-free write of the tile's segment (callers looping over tiles sync
// before the next tile zeroes the segment).  CLS: band class (see
// band_class), or CLS_LONG; the spectrum inputs at other positions are not
// formed.  SMEMD: d lives in shared memory (batches; see inverse_weights).
template <int NF, bool NARROW, int CLS = 0, bool SMEMD = false>
__device__ __forceinline__ void inverse_tile(const SstDev &d, const float2 *__restrict__ T, float *__restrict__ partial,
                                             int64_t tile, float4 *smem4, int tid) {
    using C = Cfg<NF>;
    using TP = InvTaps<NARROW>;
    constexpr int TPF = C::TPF;
    constexpr int NS = NF / 16;
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    // staged rows.  Synchronous staging: Tst[f][s][q] = T_f[z q + s], q in
    // [0, nq), nq = N_r + 1 (regrouped by sub-grid).  Asynchronous staging (rows of the tile contiguous and 16-byte
    // aligned): the pair's two rows as they are in T, raw[f nbo + l], one bulk
    // copy per pair, the next pair's copy issued as soon as the current pair's
    // last spectrum is built, so it lands while that sub-grid's FFT runs.
    const int nq = d.k_hi - d.k_lo + 1;
    float2 *Tst = buf + C::BUF;
    float *seg = reinterpret_cast<float *>(Tst + 2 * d.z * nq);
    // (the frame buffer's 128 bytes of slack are at the end of the allocation)
    uint64_t *rbar = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(seg + d.seg_len) + 15) & ~(uintptr_t)15);
    const int64_t m0 = tile * d.B;
    const bool live = (TPF == NS) || tid < NS;
    const uint32_t pair_bytes = 16u * (uint32_t)d.nbo;
    const float2 *tile_rows = T + (size_t)m0 * d.nbo;
    bool async = d.trow_cap == 0 && m0 + d.B <= d.F && (reinterpret_cast<uintptr_t>(tile_rows) & 15) == 0;

    constexpr bool LONGW = CLS == CLS_LONG;
    constexpr int PC = LONGW ? 0 : CLS;   // pruning class
    int tap[TP::NACC];
    float2 om[TP::NACC];
    if constexpr (!LONGW) inverse_taps<NF, NARROW>(d, tid, tap, om);

    for (int i = tid; i < d.seg_len; i += TPF) seg[i] = 0.f;
    if (async && tid == 0) {
        mbar_init(rbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (async && tid == 0) {
        mbar_expect_tx(rbar, pair_bytes);
        if (!(d.test_withhold && tile == 0)) bulk_g2s(Tst, tile_rows, pair_bytes, rbar);
    }

    for (int pr = 0; pr < d.B / 2; ++pr) {
        const int64_t a = m0 + 2 * pr, b = a + 1;
        if (a >= d.F) break;
        const bool hasb = b < d.F;
        if (async) {
            // this pair's rows: bounded wait; if it ever expired, wait once more
            // (so no copy is left in flight) and stage the rest synchronously
            int ok = 1;
            if (tid == 0) {
                ok = mbar_wait(rbar, (uint32_t)(pr & 1)) ? 1 : 0;
                if (!ok) {
                    const bool landed = mbar_wait(rbar, (uint32_t)(pr & 1));
                    if (d.status) atomicOr(d.status, SST_DEV_WAIT_EXPIRED | (landed ? 0u : SST_DEV_COPY_LOST));
                }
            }
            ok = __syncthreads_and(ok);
            if (!ok) async = false;
        }
        // synchronous staging: both rows (contiguous in T), regrouped by sub-grid
        // zone centres of the pair (component recovery only)
        const int za = d.zone ? d.zone[a] : 0;
        const int zb = d.zone ? (hasb ? d.zone[b] : -1) : 0;
        for (int f = 0; f < 2 && !async; ++f) {
            const float2 *src = T + (size_t)trow_of(d, a + f) * d.nbo;
            const bool have = f == 0 || hasb;
            for (int q = tid; q < nq; q += TPF) {
                for (int s = 0; s < d.z; ++s) {
                    const int l = d.z * q + s;
                    const bool keep = !d.zone || in_zone(l, f ? zb : za, d.zone_hw);
                    Tst[(f * d.z + s) * nq + q] = (have && l < d.nbo && keep) ? __ldg(&src[l]) : make_float2(0.f, 0.f);
                }
            }
        }
        __syncthreads();
        if (async && d.zone) {   // (block-uniform) rows as copied: clear what lies outside the zones
            for (int i = tid; i < 2 * d.nbo; i += TPF) {
                const int f = i >= d.nbo ? 1 : 0;
                if (!in_zone(i - f * d.nbo, f ? zb : za, d.zone_hw)) Tst[i] = make_float2(0.f, 0.f);
            }
            __syncthreads();
        }

        float2 racc[TP::NACC];
        // sub-grids in descending order, for the Horner accumulation
        for (int s = d.z - 1; s >= 0; --s) {
            const int sb = (s == 0) ? 0 : d.z - s;
            // element q of sub-grid s of row f: staged Tst[(f z + s) nq + q], raw Tst[f nbo + z q + s]
            const int qstride = async ? d.z : 1;
            const float2 *Ta = Tst + (async ? s : s * nq), *Tam = Tst + (async ? sb : sb * nq);
            const float2 *Tb = Tst + (async ? d.nbo + s : (d.z + s) * nq);
            const float2 *Tbm = Tst + (async ? d.nbo + sb : (d.z + sb) * nq);
            inverse_first_pass<NF, PC>(d, Ta, Tam, Tb, Tbm, qstride, s, buf, tid);
            __syncthreads();
            // the pair's rows are read for the last time above: fetch the next pair's
            if (async && s == 0 && tid == 0 && 2 * (pr + 1) < d.B) {
                mbar_expect_tx(rbar, pair_bytes);
                bulk_g2s(Tst, tile_rows + (size_t)2 * (pr + 1) * d.nbo, pair_bytes, rbar);
            }
            fft_mid<NF, TPF, true>(buf, d.tw, tid);
            float2 v[16];
            fft_out<NF, TPF, true>(buf, d.tw, tid, v);
            if constexpr (LONGW)
                inverse_long_sub<NF>(d, seg, (int)(a - m0) * d.hop + d.M, hasb, v, s, tid, live);
            else if (live)
                inverse_accumulate<NF, NARROW>(d, racc, v, om, tap, tid, s == d.z - 1);
        }
        // overlap-add a, then b (ascending frame order at every sample)
        const int oa = (int)(a - m0) * d.hop + d.M;
        if constexpr (LONGW) {
            (void)oa;   // (added sub-grid by sub-grid above)
        } else if constexpr (SMEMD) {
            float gw[TP::NACC];
            inverse_weights<NF, NARROW>(d, tap, gw);
            inverse_ola_w<NARROW, false>(seg, oa, tap, gw, racc);
            __syncthreads();
            if (hasb) inverse_ola_w<NARROW, true>(seg, oa + d.hop, tap, gw, racc);
        } else {
            inverse_ola<NF, NARROW, false>(d, seg, oa, tap, racc);
            __syncthreads();
            if (hasb) inverse_ola<NF, NARROW, true>(d, seg, oa + d.hop, tap, racc);
        }
        __syncthreads();
    }
    float *out = partial + (size_t)tslot_of(d, tile) * d.seg_len;
    for (int i = tid; i < d.seg_len; i += TPF) out[i] = seg[i];
}

#define SST_INV_MINB ((512 / Cfg<NF>::TPF < 1) ? 1 : 512 / Cfg<NF>::TPF)

template <int NF, bool NARROW, int CLS = 0>
__global__ void __launch_bounds__(Cfg<NF>::TPF, SST_INV_MINB)
k_inverse(SstDev d, const float2 *__restrict__ T, float *__restrict__ partial) {
    extern __shared__ float4 smem4[];
    inverse_tile<NF, NARROW, CLS>(d, T, partial, blockIdx.x, smem4, threadIdx.x);
}

__device__ __forceinline__ float recip_norm(const SstDev &d, int64_t p) {
    if (p < d.EL) return d.rD_left[p];
    if (p >= d.ER) return d.rD_right[p - d.ER];
    return d.rD_per[p % d.hop];
}

// xhat[p] = (sum over the tiles whose segment covers p, in tile order) / D[p]
__device__ __forceinline__ float finalize_value(const SstDev &d, const float *__restrict__ partial, int64_t p) {
    const int64_t BH = (int64_t)d.B * d.hop;
    const int64_t num = p + d.M - d.seg_len + 1;
    const int64_t tlo = num <= 0 ? 0 : (num + BH - 1) / BH;
    int64_t thi = (p + d.M) / BH;
    if (thi > d.ntiles - 1) thi = d.ntiles - 1;
    float s = 0.f;
    for (int64_t t = tlo; t <= thi; ++t) s += partial[tslot_of(d, t) * d.seg_len + (p + d.M - t * BH)];
    return s * recip_norm(d, p);
}

__global__ void k_finalize(SstDev d, const float *__restrict__ partial, float *__restrict__ xhat);

// ---------------------------------------------------------------------------
// Fused forward + inverse (sst_forward_inverse without a TFR output): one CTA
// per inverse tile of B frames.  Per pair of frames (a, b) the forward of each
// (as k_forward, MODE_TROW) leaves its T row in shared memory, and the pair is
// inverted from those rows exactly as inverse_tile does from rows staged by
// its bulk copy (Eq. 25, the z sub-grid IFFTs), then overlap-added into the
// tile's segment (Eq. 26; k_finalize sums segments and applies 1 / D).  T
// never reaches global memory.  Shared memory: the frame buffer, the T
// accumulators (whose first half holds row b while the pair is inverted), row
// a, the band mirrors (CLS > 0), the segment and, where row b is longer than
// the frame buffer, the region it is read out into.  With the one-pass
// threshold (d.fused_count set) the sources between the two bounds are
// recorded per tile instead of accumulated (k_fused_settle adds the kept ones
// later) and the exact max |S^g|^2 goes to d.spec.ctl[0].
// ---------------------------------------------------------------------------
template <int NF, bool NARROW, int CLS>
__device__ __forceinline__ void inverse_pair_rows(const SstDev &d, const float2 *__restrict__ rowA,
                                                  const float2 *__restrict__ rowB, float2 *buf, int tid,
                                                  const int (&tap)[InvTaps<NARROW>::NACC],
                                                  const float2 (&om)[InvTaps<NARROW>::NACC],
                                                  float2 (&racc)[InvTaps<NARROW>::NACC]) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    constexpr int NS = NF / 16;
    const bool live = (TPF == NS) || tid < NS;
    for (int s = d.z - 1; s >= 0; --s) {
        const int sb = (s == 0) ? 0 : d.z - s;
        // element q of sub-grid s of a row: row[z q + s]
        inverse_first_pass<NF, CLS>(d, rowA + s, rowA + sb, rowB + s, rowB + sb, d.z, s, buf, tid);
        __syncthreads();
        fft_mid<NF, TPF, true>(buf, d.tw, tid);
        float2 v[16];
        fft_out<NF, TPF, true>(buf, d.tw, tid, v);
        if (live) inverse_accumulate<NF, NARROW>(d, racc, v, om, tap, tid, s == d.z - 1);
    }
}

// The pair's sub-grid inverses for a window longer than NF + 1, added to the
// segment as they come (inverse_long_sub).
template <int NF>
__device__ __forceinline__ void inverse_pair_rows_long(const SstDev &d, const float2 *__restrict__ rowA,
                                                       const float2 *__restrict__ rowB, float2 *buf, int tid,
                                                       float *seg, int oa, bool hasb) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    constexpr int NS = NF / 16;
    const bool live = (TPF == NS) || tid < NS;
    for (int s = d.z - 1; s >= 0; --s) {
        const int sb = (s == 0) ? 0 : d.z - s;
        inverse_first_pass<NF, 0>(d, rowA + s, rowA + sb, rowB + s, rowB + sb, d.z, s, buf, tid);
        __syncthreads();
        fft_mid<NF, TPF, true>(buf, d.tw, tid);
        float2 v[16];
        fft_out<NF, TPF, true>(buf, d.tw, tid, v);
        inverse_long_sub<NF>(d, seg, oa, hasb, v, s, tid, live);
    }
}

// bytes of the fused kernel's shared memory (layout in k_fused)
__host__ __device__ __forceinline__ size_t fused_smem_bytes(size_t smem_frame, int nb, int nbo, int seg_len, int cls) {
    size_t o = smem_frame;                         // frame buffer (+ slack)
    o += tacc_bytes(nbo);                          // accumulators; row b in their first half
    o += ((size_t)8 * nbo + 15) & ~(size_t)15;     // row a
    if (cls > 0) o += mirror_bytes(nb);            // band mirrors
    o += (4 * (size_t)seg_len + 15) & ~(size_t)15; // overlap-add segment
    // row b is read out into the frame buffer, or, where it does not fit there
    // (small Nf with a wide band and subdivision), into a region of its own
    if ((size_t)8 * nbo > smem_frame - 128) o += ((size_t)8 * nbo + 15) & ~(size_t)15;
    return o;
}

template <int NF, bool NARROW, int CLS>
__global__ void __launch_bounds__(Cfg<NF>::TPF, SST_INV_MINB)
k_fused(SstDev d, const float *__restrict__ x, const SstScalars *__restrict__ sc, float *__restrict__ partial) {
    using C = Cfg<NF>;
    using TP = InvTaps<NARROW>;
    constexpr int TPF = C::TPF;
    constexpr bool LONGW = CLS == CLS_LONG;   // a window longer than NF + 1
    constexpr int PC = LONGW ? 0 : CLS;       // pruning class
    extern __shared__ float4 smem4[];
    const int tid = threadIdx.x;
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem4) + 2 * C::BUF + 32;
    const int stride = tacc_stride(d.nbo);
    float2 *rowB = reinterpret_cast<float2 *>(acc);   // row b, in the accumulators' first half
    float2 *rowA = reinterpret_cast<float2 *>(acc + 4 * stride);
    char *after = reinterpret_cast<char *>(rowA) + ((8 * (size_t)d.nbo + 15) & ~(size_t)15);
    float2 *mz = reinterpret_cast<float2 *>(after);
    float *seg = reinterpret_cast<float *>(after + (PC > 0 ? mirror_bytes(d.nb) : 0));
    float2 *rowT = d.nbo <= C::BUF ? buf
                                   : reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(seg + d.seg_len) + 15) &
                                                                ~(uintptr_t)15);
    __shared__ int ndef;   // sources recorded for the settling pass (one-pass threshold)
    if (d.gate && *d.gate == 0u) return;
    FwdScale fs = fwd_scale(d, sc, true);
    const bool spec = d.fused_count != nullptr;
    if (spec) {
        fs.gamma2 = sc->g_lb2;
        fs.g_ub2 = sc->g_ub2;
    }
    float vmax = 0.f;
    const int64_t tile = d.tile0 + blockIdx.x;
    const int64_t m0 = tile * d.B;

    for (int i = tid; i < 4 * stride; i += TPF) acc[i] = 0u;
    for (int i = tid; i < d.seg_len; i += TPF) seg[i] = 0.f;
    if (tid == 0) ndef = 0;
    // (the first barrier inside the forward orders these before any use)

    for (int pr = 0; pr < d.B / 2; ++pr) {
        const int64_t a = m0 + 2 * pr, b = a + 1;
        if (a >= d.F) break;
        const bool hasb = b < d.F;
        // forward of a: its row into rowA (the accumulators are cleared on the way)
        forward_frame<NF, MODE_TROW, PC>(d, x, fs, rowA, nullptr, a, buf, acc, tid, nullptr, &ndef, &vmax,
                                         nullptr, mz);
        // forward of b: its row into the frame buffer (free once the frame's
        // bins are read; a region of its own where the row is longer than
        // the buffer), then moved into the accumulators' first half
        if (hasb) {
            forward_frame<NF, MODE_TROW, PC>(d, x, fs, rowT, nullptr, b, buf, acc, tid, nullptr, &ndef, &vmax,
                                             nullptr, mz);
        } else {
            __syncthreads();
            for (int l = tid; l < d.nbo; l += TPF) rowT[l] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int l = tid; l < d.nbo; l += TPF) rowB[l] = rowT[l];
        __syncthreads();

        if constexpr (LONGW) {
            inverse_pair_rows_long<NF>(d, rowA, rowB, buf, tid, seg, (int)(a - m0) * d.hop + d.M, hasb);
        } else {
            int tap[TP::NACC];
            float2 om[TP::NACC];
            inverse_taps<NF, NARROW>(d, tid, tap, om);
            float2 racc[TP::NACC];
            inverse_pair_rows<NF, NARROW, CLS>(d, rowA, rowB, buf, tid, tap, om, racc);
            // overlap-add a, then b (ascending frame order at every sample)
            const int oa = (int)(a - m0) * d.hop + d.M;
            inverse_ola<NF, NARROW, false>(d, seg, oa, tap, racc);
            __syncthreads();
            if (hasb) inverse_ola<NF, NARROW, true>(d, seg, oa + d.hop, tap, racc);
        }
        // the accumulators' first half held row b: clear it for the next pair
        // (ordered before its atomics by the barriers inside the next forward)
        for (int i = tid; i < 2 * stride; i += TPF) acc[i] = 0u;
        __syncthreads();
    }
    float *out = partial + (size_t)tslot_of(d, tile) * d.seg_len;
    for (int i = tid; i < d.seg_len; i += TPF) out[i] = seg[i];
    if (spec) {
        vmax = warp_max(vmax);
        if ((tid & 31) == 0 && vmax > 0.f) atomicMax(&d.spec.ctl[0], __float_as_uint(vmax));
        if (tid == 0) {
            d.fused_count[tile] = ndef < d.fused_cap ? ndef : d.fused_cap;
            if (ndef > 0) atomicAdd(&d.spec.ctl[5], (unsigned)ndef);   // (threshold statistics)
        }
    }
}

// ---------------------------------------------------------------------------
// Batched kernels: persistent CTAs walk a table of work items (BatchItem) of
// many channels that share this NF.  Each item's SstDev is copied into
// shared memory first; the per-unit bodies are the single-plan ones.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_chan(SstDev &sd, const BatchChan *__restrict__ ch, int c, int tid, int nthr) {
    const int *src = reinterpret_cast<const int *>(&ch[c].d);
    int *dst = reinterpret_cast<int *>(&sd);
    for (int i = tid; i < (int)(sizeof(SstDev) / sizeof(int)); i += nthr) dst[i] = src[i];
}

// a channel descriptor this NF's kernels can run (guards every loop bound
// against a corrupt table: such items are skipped)
template <int NF> __device__ __forceinline__ bool chan_ok(const SstDev &d) {
    return d.nf == NF && d.z >= 1 && d.z <= 16 && d.B >= 2 && d.B <= (1 << 20) && d.hop >= 1 && d.L >= 3 &&
           d.L <= SST_MAX_L && d.n >= 1 && d.F >= 1 && d.nbo >= 1 && d.nb >= 1 && d.seg_len >= d.L;
}

template <int NF>
__global__ void __launch_bounds__(Cfg<NF>::TPF, SST_ABSMAX_MINB)
k_absmax_batch(const BatchChan *__restrict__ ch, const BatchItem *__restrict__ items, int nitems,
               float *__restrict__ partial) {
    using C = Cfg<NF>;
    __shared__ SstDev sd;
    __shared__ float red[32];
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        load_chan(sd, ch, w.chan, tid, C::TPF);
        __syncthreads();
        const float *x = ch[w.chan].x;
        float best = 0.f;
        if (!chan_ok<NF>(sd)) {
        } else if (sd.relative) {
            for (int64_t qq = w.begin; qq < w.end; ++qq) best = absmax_quad<NF>(sd, x, qq, buf, tid, best);
        } else {
            for (int64_t p = w.begin + tid; p < w.end; p += C::TPF) best = fmaxf(best, fabsf(x[p]));
        }
        best = block_max<C::NWARP>(best, red, tid);
        if (tid == 0) partial[it] = best;
    }
}

// a channel the kernels of pruning class CLS may run: a half-length window
// and a band of class 1 .. CLS (class 1's positions are a subset of class 2's);
// CLS_LONG: a window longer than NF + 1
template <int NF, int CLS> __device__ __forceinline__ bool class_ok(const SstDev &d) {
    if constexpr (CLS == 0) {
        return true;
    } else if constexpr (CLS == CLS_LONG) {
        return d.L > NF + 1;
    } else {
        const int c = band_class(NF, FftPlan<NF>::R1, d.k_hi);
        return d.L <= NF / 2 + 1 && c >= 1 && c <= CLS;
    }
}

// CLS: the pruning class of every channel in the group (the band mirrors
// then follow the accumulators, sized for max_nbo bins)
template <int NF, int CLS = 0>
__global__ void __launch_bounds__(Cfg<NF>::TPF, Cfg<NF>::MINB)
k_forward_batch(const BatchChan *__restrict__ ch, const BatchItem *__restrict__ items, int nitems, int max_nbo) {
    using C = Cfg<NF>;
    __shared__ SstDev sd;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem4) + 2 * C::BUF + 32;
    float2 *mz = reinterpret_cast<float2 *>(acc + 4 * tacc_stride(max_nbo));
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * tacc_stride(max_nbo); i += C::TPF) acc[i] = 0u;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        __syncthreads();   // previous item done with sd
        load_chan(sd, ch, w.chan, tid, C::TPF);
        __syncthreads();
        const BatchChan &c = ch[w.chan];
        if (!chan_ok<NF>(sd) || sd.nbo > max_nbo || w.end > sd.F || !class_ok<NF, CLS>(sd)) continue;
        const FwdScale fs = fwd_scale(sd, c.sc, true);
        for (int64_t m = w.begin; m < w.end; ++m)
            forward_frame<NF, MODE_T, CLS>(sd, c.x, fs, c.T, nullptr, m, buf, acc, tid, nullptr, nullptr, nullptr,
                                           nullptr, mz);
    }
}

template <int NF, bool NARROW, int CLS = 0>
__global__ void __launch_bounds__(Cfg<NF>::TPF, SST_INV_MINB)
k_inverse_batch(const BatchChan *__restrict__ ch, const BatchItem *__restrict__ items, int nitems) {
    using C = Cfg<NF>;
    __shared__ SstDev sd;
    extern __shared__ float4 smem4[];
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        __syncthreads();   // previous tile's segment written out, sd free
        load_chan(sd, ch, w.chan, tid, C::TPF);
        __syncthreads();
        if (!chan_ok<NF>(sd) || w.begin >= sd.ntiles || !class_ok<NF, CLS>(sd)) continue;
        inverse_tile<NF, NARROW, CLS, true>(sd, ch[w.chan].T, ch[w.chan].ola, w.begin, smem4, tid);
    }
}

// per-channel reductions of the batched pre-pass (one CTA per channel)
__global__ void k_gamma_batch(BatchChan *__restrict__ ch, int nchan, const float *__restrict__ partial);
// xhat of every channel (items: sample ranges)
__global__ void k_finalize_batch(const BatchChan *__restrict__ ch, const BatchItem *__restrict__ items, int nitems);

}  // namespace sst
