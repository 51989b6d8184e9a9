// Kernels of the downsampled synchrosqueezing transform, templated on the
// DFT length NF.  One CTA of TPF threads works on one frame (forward) or one
// pair of frames (threshold pre-pass, inverse) at a time.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sst_dev.h"
#include "sst_fft.cuh"

namespace sst {

template <int NF> struct Cfg {
    static constexpr int TPF = (NF / 16 < 32) ? 32 : NF / 16;  // threads per CTA
    static constexpr int PPT = NF / TPF;                          // FFT points per thread
    static constexpr int BUF = padded_len(NF);                    // float2 per frame buffer
    static constexpr int KMAX = (NF / 2 + 1 + TPF - 1) / TPF;     // band bins per thread
    static constexpr int NMAX = (NF + 1 + TPF - 1) / TPF;         // window taps per thread (L <= NF+1)
    static constexpr int NWARP = TPF / 32;
};

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

// Gather frame m (or the pair m, m2 into re/im) with window folding mod NF:
// buf[p] = sum_{j = p mod NF, |j| <= M} x[m hop + j] * win[j]   (Eq. 8-9).
// PAIR = false: win = (g, s g'), value = x (g + i s g'); s is a power of two
//               that equalises the two halves' norms (so neither half's FFT
//               rounding swamps the other) and is undone exactly afterwards
// PAIR = true : value = (x_m + i x_m2) g
template <int NF, bool PAIR>
__device__ __forceinline__ void gather_frame(float2 *buf, const SstDev &d, const float *__restrict__ x,
                                             int64_t m, int64_t m2, bool has2, int tid) {
    constexpr int TPF = Cfg<NF>::TPF;
    const int64_t c1 = m * d.hop, c2 = m2 * d.hop;
#pragma unroll 4
    for (int i = 0; i < Cfg<NF>::PPT; ++i) {
        const int p = tid + i * TPF;
        float2 acc = make_float2(0.f, 0.f);
        const int jmin = p - NF * ((p + d.M) / NF);
        for (int j = jmin; j <= d.M; j += NF) {
            const float2 w = __ldg(&d.win[j + d.M]);
            const int64_t s1 = c1 + j;
            const float x1 = (s1 >= 0 && s1 < d.n) ? __ldg(&x[s1]) : 0.f;
            if (!PAIR) {
                acc.x = fmaf(x1, w.x, acc.x);
                acc.y = fmaf(x1, w.y, acc.y);
            } else {
                const int64_t s2 = c2 + j;
                const float x2 = (has2 && s2 >= 0 && s2 < d.n) ? __ldg(&x[s2]) : 0.f;
                acc.x = fmaf(x1, w.x, acc.x);
                acc.y = fmaf(x2, w.x, acc.y);
            }
        }
        buf[padded(p)] = acc;
    }
}

// ---------------------------------------------------------------------------
// Threshold pre-pass: max |S^g|^2 over in-band bins of every frame.  Two real
// frames share one complex FFT: Z = FFT((x_a + i x_b) g), S_a = (Z[k] +
// conj Z[-k]) / 2, S_b = (Z[k] - conj Z[-k]) / 2i.  One partial max per CTA.
// ---------------------------------------------------------------------------
template <int NF>
__global__ void __launch_bounds__(Cfg<NF>::TPF)
k_absmax(SstDev d, const float *__restrict__ x, float *__restrict__ partial) {
    using C = Cfg<NF>;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    float *red = reinterpret_cast<float *>(buf + C::BUF);
    const int tid = threadIdx.x;
    const int64_t npairs = (d.F + 1) / 2;
    float best = 0.f;
    for (int64_t q = blockIdx.x; q < npairs; q += gridDim.x) {
        const int64_t a = 2 * q, b = a + 1;
        const bool hasb = b < d.F;
        gather_frame<NF, true>(buf, d, x, a, b, hasb, tid);
        __syncthreads();
        fft<NF, C::TPF, false>(buf, d.tw, tid);
        for (int kk = tid; kk < d.nb; kk += C::TPF) {
            const int k = d.k_lo + kk;
            const float2 zk = buf[padded(k)];
            const float2 zm = buf[padded((NF - k) & (NF - 1))];
            const float ar = 0.5f * (zk.x + zm.x), ai = 0.5f * (zk.y - zm.y);
            best = fmaxf(best, ar * ar + ai * ai);
            if (hasb) {
                const float br = 0.5f * (zk.y + zm.y), bi = 0.5f * (zm.x - zk.x);
                best = fmaxf(best, br * br + bi * bi);
            }
        }
        __syncthreads();
    }
    best = block_max<C::NWARP>(best, red, tid);
    if (tid == 0) partial[blockIdx.x] = best;
}

// gamma^2 = frac^2 * max over partials; also stores max |S^g|
__global__ void k_gamma(const float *__restrict__ partial, int count, float frac2,
                        float *__restrict__ gamma2_out, float *__restrict__ maxv_out);

// ---------------------------------------------------------------------------
// Forward: per frame, packed FFT of x (g + i g'), Hermitian split into S^g and
// S^g' for the band bins, IF estimate, threshold, destination, and the
// deterministic per-frame accumulation of T in shared memory.
//   MODE_T   : T rows (F x nbo complex)
//   MODE_STFT: S^g, S^g' rows (F x nb complex each), no threshold
//   MODE_MAP : omega (F x nb float) and dest (F x nb int32)
// The T sum is exact: every contribution is scaled by a per-frame power of
// two 2^e, chosen so that any sum of the frame's terms stays below 2^62, and
// converted to int64 (exactly, for all but sub-2^-39-relative terms);
// shared-memory 64-bit integer adds are order independent, so the rounded
// result does not depend on thread scheduling.
// ---------------------------------------------------------------------------
enum { MODE_T = 0, MODE_STFT = 1, MODE_MAP = 2 };

template <int NF, int MODE>
__global__ void __launch_bounds__(Cfg<NF>::TPF)
k_forward(SstDev d, const float *__restrict__ x, const float *__restrict__ gamma2_dev,
          float2 *__restrict__ out0, void *__restrict__ out1) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    float *red = reinterpret_cast<float *>(buf + C::BUF);
    // after the frame buffer (BUF float2 = BUF x 8 bytes) and 128 bytes of reduction scratch
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(smem4) + C::BUF + 16;
    const int tid = threadIdx.x;
    const float gamma2 = d.relative ? __ldg(gamma2_dev) : d.gamma2_abs;

    if (MODE == MODE_T)
        for (int i = tid; i < 2 * d.nbo; i += TPF) acc[i] = 0ull;
    // (the first __syncthreads below orders this before any atomic)

    for (int64_t m = blockIdx.x; m < d.F; m += gridDim.x) {
        gather_frame<NF, false>(buf, d, x, m, 0, false, tid);
        __syncthreads();
        fft<NF, TPF, false>(buf, d.tw, tid);

        float2 Vv[C::KMAX];
        int li[C::KMAX];
        float maxc = 0.f;
#pragma unroll
        for (int i = 0; i < C::KMAX; ++i) {
            const int kk = tid + i * TPF;
            li[i] = -1;
            Vv[i] = make_float2(0.f, 0.f);
            if (kk < d.nb) {
                const int k = d.k_lo + kk;
                const float2 zk = buf[padded(k)];
                const float2 zm = buf[padded((NF - k) & (NF - 1))];
                const float2 V = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                const float2 Vd = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
                const size_t o = (size_t)m * d.nb + kk;
                if (MODE == MODE_STFT) {
                    out0[o] = V;
                    reinterpret_cast<float2 *>(out1)[o] = make_float2(Vd.x * d.dscale, Vd.y * d.dscale);
                    continue;
                }
                const float mag2 = V.x * V.x + V.y * V.y;
                // reassignment offset in bins: -(Nf / 2 pi) Im(S^g' / S^g)   (Eq. 13, 36)
                const float delta = -d.c_if * ((Vd.y * V.x - Vd.x * V.y) / mag2);
                int l = -1;
                if (mag2 > gamma2) {
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
                    continue;
                }
                li[i] = l;
                Vv[i] = V;
                if (l >= 0) maxc = fmaxf(maxc, fmaxf(fabsf(V.x), fabsf(V.y)));
            }
        }
        if (MODE != MODE_T) {
            __syncthreads();  // buf reads done before the next gather
            continue;
        }
        maxc = block_max<C::NWARP>(maxc, red, tid);  // also orders buf reads before next gather
        int e = 0;
        if (maxc > 0.f) {
            int ex;
            frexpf(maxc, &ex);  // maxc < 2^ex
            e = 62 - ex - d.log2_nb;
#pragma unroll
            for (int i = 0; i < C::KMAX; ++i) {
                if (li[i] >= 0) {
                    const long long qr = __float2ll_rn(ldexpf(Vv[i].x, e));
                    const long long qi = __float2ll_rn(ldexpf(Vv[i].y, e));
                    atomicAdd(&acc[2 * li[i]], (unsigned long long)qr);
                    atomicAdd(&acc[2 * li[i] + 1], (unsigned long long)qi);
                }
            }
        }
        __syncthreads();
        float2 *Trow = out0 + (size_t)m * d.nbo;
        for (int l = tid; l < d.nbo; l += TPF) {
            const long long ar = (long long)acc[2 * l], ai = (long long)acc[2 * l + 1];
            Trow[l] = make_float2(ldexpf(__ll2float_rn(ar), -e), ldexpf(__ll2float_rn(ai), -e));
            acc[2 * l] = 0ull;
            acc[2 * l + 1] = 0ull;
        }
        // the zeroing above is ordered before the next frame's atomics by the
        // __syncthreads inside the next gather/FFT
    }
}

// ---------------------------------------------------------------------------
// Inverse, one CTA per tile of B consecutive frames (B even), frames taken in
// pairs (a, b = a + 1).  For a pair, r_a + i r_b comes out of z complex
// inverse FFTs of length NF: sub-grid s (fine bins l = z q + s) is placed at
// coarse bin k_lo + q together with the Hermitian image of sub-grid
// (z - s) mod z, and the result is multiplied by exp(i 2 pi s j / (z NF))
// (Eq. 25, with the zNf-point zero-padded inverse of Sec. 2.5 split into its
// z interleaved sub-grids).  The windowed frames are overlap-added into a
// shared-memory segment in ascending frame order, written to the partial
// buffer, and k_finalize sums overlapping segments in tile order and applies
// 1 / D[p] (Eq. 26).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 tfr_value(const float2 *__restrict__ Trow, const SstDev &d, int k, int s,
                                            int nf) {
    // w_l T[l] for the fine bin l = z (k - k_lo) + s, zero outside the grid
    const int q = k - d.k_lo;
    if (q < 0 || q > d.k_hi - d.k_lo) return make_float2(0.f, 0.f);
    const int l = d.z * q + s;
    if (l >= d.nbo) return make_float2(0.f, 0.f);
    float2 t = __ldg(&Trow[l]);
    if (s == 0 && (k == 0 || 2 * k == nf)) t = cscale(t, 0.5f);
    return t;
}

template <int NF>
__global__ void __launch_bounds__(Cfg<NF>::TPF)
k_inverse(SstDev d, const float2 *__restrict__ T, float *__restrict__ partial) {
    using C = Cfg<NF>;
    constexpr int TPF = C::TPF;
    extern __shared__ float4 smem4[];
    float2 *buf = reinterpret_cast<float2 *>(smem4);
    float *seg = reinterpret_cast<float *>(buf + C::BUF);
    const int tid = threadIdx.x;
    const int64_t tile = blockIdx.x;
    const int64_t m0 = tile * d.B;
    const float cnorm = 1.0f / (float)NF;
    const int G = d.z * NF;

    for (int i = tid; i < d.seg_len; i += TPF) seg[i] = 0.f;

    for (int pr = 0; pr < d.B / 2; ++pr) {
        const int64_t a = m0 + 2 * pr, b = a + 1;
        if (a >= d.F) break;
        const bool hasb = b < d.F;
        const float2 *Ta = T + (size_t)a * d.nbo;
        const float2 *Tb = T + (size_t)(hasb ? b : a) * d.nbo;
        float2 racc[C::NMAX];
#pragma unroll
        for (int i = 0; i < C::NMAX; ++i) racc[i] = make_float2(0.f, 0.f);

        for (int s = 0; s < d.z; ++s) {
            const int sb = (s == 0) ? 0 : d.z - s;
            const int dl = (s == 0) ? 0 : 1;
            // Y_s[k] = (1/NF) (X_a,s[k] + conj X_a,sb[-k-dl] + i (X_b,s[k] + conj X_b,sb[-k-dl]))
#pragma unroll 4
            for (int i = 0; i < C::PPT; ++i) {
                const int k = tid + i * TPF;
                const int km = (NF - k - dl) & (NF - 1);
                float2 xa = tfr_value(Ta, d, k, s, NF);
                float2 xam = tfr_value(Ta, d, km, sb, NF);
                float2 y = make_float2(xa.x + xam.x, xa.y - xam.y);
                if (hasb) {
                    const float2 xb = tfr_value(Tb, d, k, s, NF);
                    const float2 xbm = tfr_value(Tb, d, km, sb, NF);
                    // i * (xb + conj xbm)
                    y.x -= xb.y - xbm.y;
                    y.y += xb.x + xbm.x;
                }
                buf[padded(k)] = cscale(y, cnorm);
            }
            __syncthreads();
            fft<NF, TPF, true>(buf, d.tw, tid);
#pragma unroll
            for (int i = 0; i < C::NMAX; ++i) {
                const int t = tid + i * TPF;  // t = j + M
                if (t < d.L) {
                    const int j = t - d.M;
                    const float2 yv = buf[padded(j & (NF - 1))];
                    if (s == 0) {
                        racc[i] = cadd(racc[i], yv);
                    } else {
                        int qi = (s * j) % G;
                        if (qi < 0) qi += G;
                        racc[i] = cadd(racc[i], cmul(yv, __ldg(&d.twz[qi])));
                    }
                }
            }
            __syncthreads();
        }
        // overlap-add a, then b (ascending frame order at every sample)
        const int oa = (int)(a - m0) * d.hop;
#pragma unroll
        for (int i = 0; i < C::NMAX; ++i) {
            const int t = tid + i * TPF;
            if (t < d.L) seg[oa + t] += __ldg(&d.g[t]) * racc[i].x;
        }
        __syncthreads();
        if (hasb) {
            const int ob = oa + d.hop;
#pragma unroll
            for (int i = 0; i < C::NMAX; ++i) {
                const int t = tid + i * TPF;
                if (t < d.L) seg[ob + t] += __ldg(&d.g[t]) * racc[i].y;
            }
            __syncthreads();
        }
    }
    float *out = partial + (size_t)tile * d.seg_len;
    for (int i = tid; i < d.seg_len; i += TPF) out[i] = seg[i];
}

__global__ void k_finalize(SstDev d, const float *__restrict__ partial, float *__restrict__ xhat);

}  // namespace sst
