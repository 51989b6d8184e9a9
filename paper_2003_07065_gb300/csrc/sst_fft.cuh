// Shared-memory Stockham FFT for one frame of NF complex float32 points,
// executed cooperatively by TPF >= NF/16 threads of a CTA.
//
// Layout: the frame lives in shared memory as float2 with one pad element
// after every 16 (index i -> i + i/16), which keeps the stride-16 scatter of
// the first radix-16 pass free of bank conflicts.  Each pass loads R points
// per butterfly into registers, applies the Stockham twiddles
// W_{Ns R}^{r k} = exp(-2 pi i r k / (Ns R)), runs a radix-R DFT in registers
// and stores the results in autosorted order.  Passes: one radix 2, 4, 8 or
// 16 pass, then radix-16 passes; output in natural order.  The first and last
// passes are also offered with their inputs / outputs in registers so that
// kernels can fuse the frame gather into the first and their epilogue into
// the last.
//
// Twiddles: a table built in FP64 on the host and rounded holds, for each
// radix-16 pass of span Ns (Ns = R1, 16 R1, ..., NF/16), the four rows
// W^{m k}, m = 1, 2, 4, 8, k in [0, Ns) (k fastest, so a warp's load is
// contiguous), starting at entry 4 (Ns - R1) / 15.  A butterfly loads its four
// values and forms the other eleven powers with at most three complex
// products, so every twiddle is within a few ulp of the exact value.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sst {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 rot90(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

__host__ __device__ constexpr int padded(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }

// Padded index of element i0 + r STRIDE given p0 = padded(i0).  When STRIDE is
// a multiple of 16 the pad count grows by exactly STRIDE / 16 per step, so
// the address is p0 plus a compile-time constant (an immediate offset on the
// shared-memory access, no per-element index arithmetic).
template <int STRIDE> __device__ __forceinline__ int padded_at(int i0, int p0, int r) {
    if constexpr (STRIDE % 16 == 0) return p0 + r * (STRIDE + STRIDE / 16);
    else return padded(i0 + r * STRIDE);
}

// sqrt(1/2), cos(pi/8), sin(pi/8)
#define SST_R2 0.70710678118654752440f
#define SST_C8 0.92387953251128675613f
#define SST_S8 0.38268343236508977173f

template <bool INV> __device__ __forceinline__ void dft2(float2 &a0, float2 &a1) {
    float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV> __device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    float2 s0 = cadd(a0, a2), d0 = csub(a0, a2);
    float2 s1 = cadd(a1, a3), d1 = rot90<INV>(csub(a1, a3));
    a0 = cadd(s0, s1);
    a2 = csub(s0, s1);
    a1 = cadd(d0, d1);
    a3 = csub(d0, d1);
}

// multiply by W8^k (forward: exp(-i pi k / 4)), k = 1, 3
template <bool INV> __device__ __forceinline__ float2 w8_1(float2 a) {
    // forward: (1 - i)/sqrt2 ; inverse: (1 + i)/sqrt2
    return INV ? make_float2(SST_R2 * (a.x - a.y), SST_R2 * (a.x + a.y))
               : make_float2(SST_R2 * (a.x + a.y), SST_R2 * (a.y - a.x));
}
template <bool INV> __device__ __forceinline__ float2 w8_3(float2 a) {
    // forward: (-1 - i)/sqrt2 ; inverse: (-1 + i)/sqrt2
    return INV ? make_float2(-SST_R2 * (a.x + a.y), SST_R2 * (a.x - a.y))
               : make_float2(SST_R2 * (a.y - a.x), -SST_R2 * (a.x + a.y));
}

// 8-point DFT: two 4-point DFTs of the even and odd samples, then W8 combine
template <bool INV> __device__ __forceinline__ void dft8(float2 *v) {
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    float2 o1 = w8_1<INV>(v[3]);
    float2 o2 = rot90<INV>(v[5]);
    float2 o3 = w8_3<INV>(v[7]);
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// multiply by W16^e for e in 0..9 (forward exp(-2 pi i e / 16))
template <bool INV, int E> __device__ __forceinline__ float2 w16(float2 a) {
    constexpr float c[10] = {1.f, SST_C8, SST_R2, SST_S8, 0.f, -SST_S8, -SST_R2, -SST_C8, -1.f, -SST_C8};
    constexpr float s[10] = {0.f, SST_S8, SST_R2, SST_C8, 1.f, SST_C8, SST_R2, SST_S8, 0.f, -SST_S8};
    // forward multiplier: c - i s ; inverse: c + i s
    if (E == 0) return a;
    if (E == 4) return rot90<INV>(a);
    const float cc = c[E], ss = INV ? s[E] : -s[E];
    return make_float2(a.x * cc - a.y * ss, a.x * ss + a.y * cc);
}

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV> __device__ __forceinline__ void dft16(float2 *v) {
    // step 1: for each n2, DFT4 over n1 of v[4 n1 + n2]; result Y[n2][k1] kept at v[4 k1 + n2]
    dft4<INV>(v[0], v[4], v[8], v[12]);
    dft4<INV>(v[1], v[5], v[9], v[13]);
    dft4<INV>(v[2], v[6], v[10], v[14]);
    dft4<INV>(v[3], v[7], v[11], v[15]);
    // step 2: twiddle Y[n2][k1] *= W16^{n2 k1}
    v[5] = w16<INV, 1>(v[5]);
    v[9] = w16<INV, 2>(v[9]);
    v[13] = w16<INV, 3>(v[13]);
    v[6] = w16<INV, 2>(v[6]);
    v[10] = w16<INV, 4>(v[10]);
    v[14] = w16<INV, 6>(v[14]);
    v[7] = w16<INV, 3>(v[7]);
    v[11] = w16<INV, 6>(v[11]);
    v[15] = w16<INV, 9>(v[15]);
    // step 3: for each k1, DFT4 over n2 of Y[n2][k1] (at v[4 k1 + n2]) -> X[k1 + 4 k2]
    dft4<INV>(v[0], v[1], v[2], v[3]);
    dft4<INV>(v[4], v[5], v[6], v[7]);
    dft4<INV>(v[8], v[9], v[10], v[11]);
    dft4<INV>(v[12], v[13], v[14], v[15]);
    // now X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4x4 index
    float2 t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

// 4-point DFT whose inputs a_i with bit i of M clear are known to be zero
// (their registers are not read).  M = 0 leaves the outputs unset: they are
// zero, and the caller treats them as such.
template <bool INV, int M> __device__ __forceinline__ void dft4m(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    if constexpr (M == 15) {
        dft4<INV>(a0, a1, a2, a3);
    } else if constexpr (M != 0) {
        constexpr bool e0 = M & 1, e1 = M & 2, e2 = M & 4, e3 = M & 8;
        const float2 zero = make_float2(0.f, 0.f);
        // s0 = a0 + a2, d0 = a0 - a2, s1 = a1 + a3, d1 = -+i (a1 - a3)
        float2 s0, d0, s1, d1;
        if constexpr (e0 && e2) { s0 = cadd(a0, a2); d0 = csub(a0, a2); }
        else if constexpr (e0) { s0 = a0; d0 = a0; }
        else if constexpr (e2) { s0 = a2; d0 = make_float2(-a2.x, -a2.y); }
        else { s0 = zero; d0 = zero; }
        if constexpr (e1 && e3) { s1 = cadd(a1, a3); d1 = rot90<INV>(csub(a1, a3)); }
        else if constexpr (e1) { s1 = a1; d1 = rot90<INV>(a1); }
        else if constexpr (e3) { s1 = a3; d1 = rot90<INV>(make_float2(-a3.x, -a3.y)); }
        else { s1 = zero; d1 = zero; }
        constexpr bool h0 = e0 || e2, h1 = e1 || e3;
        if constexpr (h0 && h1) {
            a0 = cadd(s0, s1); a2 = csub(s0, s1); a1 = cadd(d0, d1); a3 = csub(d0, d1);
        } else if constexpr (h0) {
            a0 = s0; a2 = s0; a1 = d0; a3 = d0;
        } else {
            a0 = s1; a2 = make_float2(-s1.x, -s1.y); a1 = d1; a3 = make_float2(-d1.x, -d1.y);
        }
    }
}

// 16-point DFT (as dft16) of inputs v[r] that are zero where bit r of MASK is
// clear; zero inputs are not read and the operations they would feed are
// left out (for spectra and windows that occupy part of the frame only).
template <bool INV, unsigned MASK> __device__ __forceinline__ void dft16m(float2 *v) {
    if constexpr (MASK == 0xffffu) {
        dft16<INV>(v);
    } else {
        // group n2 holds inputs r = n2, n2 + 4, n2 + 8, n2 + 12
        constexpr int G0 = ((MASK >> 0) & 1) | ((MASK >> 3) & 2) | ((MASK >> 6) & 4) | ((MASK >> 9) & 8);
        constexpr int G1 = ((MASK >> 1) & 1) | ((MASK >> 4) & 2) | ((MASK >> 7) & 4) | ((MASK >> 10) & 8);
        constexpr int G2 = ((MASK >> 2) & 1) | ((MASK >> 5) & 2) | ((MASK >> 8) & 4) | ((MASK >> 11) & 8);
        constexpr int G3 = ((MASK >> 3) & 1) | ((MASK >> 6) & 2) | ((MASK >> 9) & 4) | ((MASK >> 12) & 8);
        dft4m<INV, G0>(v[0], v[4], v[8], v[12]);
        dft4m<INV, G1>(v[1], v[5], v[9], v[13]);
        dft4m<INV, G2>(v[2], v[6], v[10], v[14]);
        dft4m<INV, G3>(v[3], v[7], v[11], v[15]);
        if constexpr (G1 != 0) { v[5] = w16<INV, 1>(v[5]); v[9] = w16<INV, 2>(v[9]); v[13] = w16<INV, 3>(v[13]); }
        if constexpr (G2 != 0) { v[6] = w16<INV, 2>(v[6]); v[10] = w16<INV, 4>(v[10]); v[14] = w16<INV, 6>(v[14]); }
        if constexpr (G3 != 0) { v[7] = w16<INV, 3>(v[7]); v[11] = w16<INV, 6>(v[11]); v[15] = w16<INV, 9>(v[15]); }
        // second step: group k1 holds Y[n2][k1] at v[4 k1 + n2], present where G(n2) != 0
        constexpr int H = (G0 ? 1 : 0) | (G1 ? 2 : 0) | (G2 ? 4 : 0) | (G3 ? 8 : 0);
        const float2 zero = make_float2(0.f, 0.f);
        dft4m<INV, H>(v[0], v[1], v[2], v[3]);
        dft4m<INV, H>(v[4], v[5], v[6], v[7]);
        dft4m<INV, H>(v[8], v[9], v[10], v[11]);
        dft4m<INV, H>(v[12], v[13], v[14], v[15]);
        if constexpr (H == 0) {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = zero;
        }
        float2 t;
        t = v[1]; v[1] = v[4]; v[4] = t;
        t = v[2]; v[2] = v[8]; v[8] = t;
        t = v[3]; v[3] = v[12]; v[12] = t;
        t = v[6]; v[6] = v[9]; v[9] = t;
        t = v[7]; v[7] = v[13]; v[13] = t;
        t = v[11]; v[11] = v[14]; v[14] = t;
    }
}

template <int R, bool INV> __device__ __forceinline__ void dft_r(float2 *v) {
    if constexpr (R == 2) dft2<INV>(v[0], v[1]);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<INV>(v);
    else dft16<INV>(v);
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

template <int NF> __host__ __device__ constexpr int first_radix() {
    return (ilog2c(NF) % 4 == 0) ? 16 : (1 << (ilog2c(NF) % 4));
}
template <int NF, int NS> __host__ __device__ constexpr int tw_offset() { return 4 * (NS - first_radix<NF>()) / 15; }

// v[r] *= W^{r k} for r = 1..15, W = exp(-+2 pi i / (16 NS)), from the four
// table rows of the pass at t (see the header)
template <bool INV>
__device__ __forceinline__ void twiddle16(float2 *v, const float2 *__restrict__ t, int NS, int k) {
    float2 w1 = __ldg(&t[k]), w2 = __ldg(&t[NS + k]), w4 = __ldg(&t[2 * NS + k]), w8 = __ldg(&t[3 * NS + k]);
    if (INV) { w1.y = -w1.y; w2.y = -w2.y; w4.y = -w4.y; w8.y = -w8.y; }
    const float2 w3 = cmul(w2, w1), w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], w5);
    v[6] = cmul(v[6], w6);
    v[7] = cmul(v[7], w7);
    v[8] = cmul(v[8], w8);
    v[9] = cmul(v[9], cmul(w8, w1));
    v[10] = cmul(v[10], cmul(w8, w2));
    v[11] = cmul(v[11], cmul(w8, w3));
    v[12] = cmul(v[12], cmul(w8, w4));
    v[13] = cmul(v[13], cmul(w8, w5));
    v[14] = cmul(v[14], cmul(w8, w6));
    v[15] = cmul(v[15], cmul(w8, w7));
}

// The fifteen twiddles W^{r k}, r = 1..15, of a radix-16 butterfly (w[0] unused)
template <bool INV>
__device__ __forceinline__ void twiddles16(float2 (&w)[16], const float2 *__restrict__ t, int NS, int k) {
    float2 w1 = __ldg(&t[k]), w2 = __ldg(&t[NS + k]), w4 = __ldg(&t[2 * NS + k]), w8 = __ldg(&t[3 * NS + k]);
    if (INV) { w1.y = -w1.y; w2.y = -w2.y; w4.y = -w4.y; w8.y = -w8.y; }
    w[1] = w1; w[2] = w2; w[4] = w4; w[8] = w8;
    w[3] = cmul(w2, w1); w[5] = cmul(w4, w1); w[6] = cmul(w4, w2); w[7] = cmul(w4, w[3]);
#pragma unroll
    for (int r = 1; r < 8; ++r) w[8 + r] = cmul(w8, w[r]);
}

// ---- several independent frames per thread (instruction-level parallelism)
// Frame f of NB lives at buf + f * BS (BS float2 apart).  Every routine below
// assumes TPF >= NF / 16 (one radix-16 butterfly per thread and pass).

// radix-16 pass with span NS > 1 on NB frames; twiddles shared by the frames
template <int NF, int TPF, int NS, bool INV, int NB, int BS>
__device__ __forceinline__ void stockham16_multi(float2 *buf, const float2 *__restrict__ tw, int tid) {
    constexpr int NBF = NF / 16;
    const bool live = (TPF == NBF) || tid < NBF;
    float2 v[NB][16];
    if (live) {
        const int p0 = padded(tid);
#pragma unroll
        for (int f = 0; f < NB; ++f)
#pragma unroll
            for (int r = 0; r < 16; ++r) v[f][r] = buf[f * BS + padded_at<NBF>(tid, p0, r)];
    }
    __syncthreads();
    if (live) {
        const int k = tid & (NS - 1);
        float2 w[16];
        twiddles16<INV>(w, tw + tw_offset<NF, NS>(), NS, k);
        const int base = (tid - k) * 16 + k;
        const int pb = padded(base);
#pragma unroll
        for (int f = 0; f < NB; ++f) {
#pragma unroll
            for (int r = 1; r < 16; ++r) v[f][r] = cmul(v[f][r], w[r]);
            dft16<INV>(v[f]);
#pragma unroll
            for (int r = 0; r < 16; ++r) buf[f * BS + padded_at<NS>(base, pb, r)] = v[f][r];
        }
    }
    __syncthreads();
}

template <int NF, int TPF, int NS, bool INV, int NB, int BS>
__device__ __forceinline__ void fft_middle_multi(float2 *buf, const float2 *__restrict__ tw, int tid) {
    if constexpr (NS < NF / 16) {
        stockham16_multi<NF, TPF, NS, INV, NB, BS>(buf, tw, tid);
        fft_middle_multi<NF, TPF, NS * 16, INV, NB, BS>(buf, tw, tid);
    }
}

// last pass of NB frames into registers (see fft_last_to_regs); ends with a barrier
template <int NF, int TPF, bool INV, int NB, int BS>
__device__ __forceinline__ void fft_last_multi(const float2 *buf, const float2 *__restrict__ tw, int tid,
                                               float2 (&v)[NB][16]) {
    constexpr int NS = NF / 16;
    if (TPF == NS || tid < NS) {
        const int p0 = padded(tid);
#pragma unroll
        for (int f = 0; f < NB; ++f)
#pragma unroll
            for (int r = 0; r < 16; ++r) v[f][r] = buf[f * BS + padded_at<NS>(tid, p0, r)];
        float2 w[16];
        twiddles16<INV>(w, tw + tw_offset<NF, NS>(), NS, tid);
#pragma unroll
        for (int f = 0; f < NB; ++f) {
#pragma unroll
            for (int r = 1; r < 16; ++r) v[f][r] = cmul(v[f][r], w[r]);
            dft16<INV>(v[f]);
        }
    }
    __syncthreads();
}

// One Stockham pass of radix R with span NS (product of earlier radices).
template <int NF, int TPF, int R, int NS, bool INV>
__device__ __forceinline__ void stockham_pass(float2 *buf, const float2 *__restrict__ tw, int tid) {
    constexpr int NBF = NF / R;                   // butterflies in this pass
    constexpr int PER = (NBF + TPF - 1) / TPF;    // butterflies per thread
    static_assert(NS == 1 || R == 16, "passes after the first are radix 16");
    float2 v[PER][R];
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        const int j = tid + b * TPF;
        if (PER * TPF == NBF || j < NBF) {
            const int p0 = padded(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = buf[padded_at<NBF>(j, p0, r)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        const int j = tid + b * TPF;
        if (PER * TPF == NBF || j < NBF) {
            const int k = j & (NS - 1);
            if constexpr (NS > 1) twiddle16<INV>(v[b], tw + tw_offset<NF, NS>(), NS, k);
            dft_r<R, INV>(v[b]);
            const int base = (j - k) * R + k;
            if constexpr (NS == 1) {
                // span 1: the R outputs j R .. j R + R - 1 share one pad block (R divides 16)
                const int pb = padded(base);
#pragma unroll
                for (int r = 0; r < R; ++r) buf[pb + r] = v[b][r];
            } else {
                const int pb = padded(base);
#pragma unroll
                for (int r = 0; r < R; ++r) buf[padded_at<NS>(base, pb, r)] = v[b][r];
            }
        }
    }
    __syncthreads();
}

// Pass plan: log2(NF) = 4a + b.  The first pass has radix R1 = 2^b (or 16
// when b = 0) and span 1; every later pass has radix 16; the last pass has
// span NF/16, so its butterfly j holds the outputs q = j + r NF/16.
template <int NF> struct FftPlan {
    static constexpr int LOG = ilog2c(NF);
    static constexpr int R1 = first_radix<NF>();
    static constexpr int NS_LAST = NF / 16;
};

// Middle passes: radix 16, spans R1, 16 R1, ..., up to (not including) NF/16.
template <int NF, int TPF, int NS, bool INV>
__device__ __forceinline__ void fft_middle(float2 *buf, const float2 *__restrict__ tw, int tid) {
    if constexpr (NS < NF / 16) {
        stockham_pass<NF, TPF, 16, NS, INV>(buf, tw, tid);
        fft_middle<NF, TPF, NS * 16, INV>(buf, tw, tid);
    }
}

// First pass from registers: butterfly j = tid + b TPF holds the inputs
// x[j + r NF/R1] in v[b][r]; the R1-point DFT is applied and the results
// stored in autosorted order (span 1: x'[j R1 + r]).  No barrier inside;
// the caller must __syncthreads() before the next pass.
// MASK (R1 = 16 only): inputs r whose bit is clear are zero and not read.
template <int NF, int TPF, bool INV, unsigned MASK = 0xffffu>
__device__ __forceinline__ void fft_first_from_regs(float2 *buf, float2 (*v)[FftPlan<NF>::R1], int tid) {
    constexpr int R1 = FftPlan<NF>::R1;
    constexpr int NBF = NF / R1;
    constexpr int PER = (NBF + TPF - 1) / TPF;
    static_assert(MASK == 0xffffu || R1 == 16, "input masks need a radix-16 first pass");
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        const int j = tid + b * TPF;
        if (PER * TPF == NBF || j < NBF) {
            if constexpr (MASK == 0xffffu) dft_r<R1, INV>(v[b]);
            else dft16m<INV, MASK>(v[b]);
            // outputs j R1 .. j R1 + R1 - 1 share one pad block (R1 divides 16)
            const int pb = padded(j * R1);
#pragma unroll
            for (int r = 0; r < R1; ++r) buf[pb + r] = v[b][r];
        }
    }
}

// Last pass into registers: butterfly j (< NF/16) loads x[j + r NF/16],
// applies W_NF^{r j}, and leaves the outputs X[j + r NF/16] in v[r].  Ends
// with a __syncthreads() (SYNC), after which buf may be reused.
template <int NF, int TPF, bool INV, bool SYNC = true>
__device__ __forceinline__ void fft_last_to_regs(const float2 *buf, const float2 *__restrict__ tw, int tid,
                                                 float2 (&v)[16]) {
    constexpr int NS = NF / 16;
    const int j = tid;
    if (TPF == NS || j < NS) {
        const int p0 = padded(j);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = buf[padded_at<NS>(j, p0, r)];
        twiddle16<INV>(v, tw + tw_offset<NF, NS>(), NS, j);
        dft16<INV>(v);
    }
    if constexpr (SYNC) __syncthreads();
}

// ---- In-place decimation in frequency, for NF = 16^P (P = 2, 3)
// Pass p combines the elements at stride ST = NF / 16^p and multiplies
// output r of butterfly s (its position within the stride) by W_{16 ST}^{s r}
// (the Stockham table of span ST); every butterfly reads and writes the same
// sixteen elements, so a pass needs one barrier (after its stores) instead of
// two.  The spectrum comes out digit-reversed in the buffer: element
// 256 k0 + 16 k1 + k2 (NF = 4096) holds X[k0 + 16 k1 + 256 k2].  The last
// pass undoes that by its choice of butterfly: thread t takes the butterfly
// of the sixteen elements 16 rev(t) .. 16 rev(t) + 15 (rev: the two hex
// digits of t swapped), whose outputs are X[t + r NF/16], the same registers
// as the Stockham last pass.  Element i lives at dpad(i) = i + i/16 + i/256,
// which keeps all three passes' accesses free of bank conflicts.
template <int NF> __host__ __device__ constexpr bool dif_ok() { return NF == 256 || NF == 4096; }
__host__ __device__ constexpr int dpad(int i) { return i + (i >> 4) + (i >> 8); }
template <int NF> __host__ __device__ constexpr int dif_len() { return dif_ok<NF>() ? dpad(NF - 1) + 1 : 0; }
template <int NF> __device__ __forceinline__ int dif_rev(int t) {
    if constexpr (NF == 4096) return ((t & 15) << 4) | (t >> 4);
    else return t;
}

// first pass from registers: butterfly j = tid (< NF/16) holds x[j + r NF/16]
// in v[r] (zero where bit r of MASK is clear); no barrier inside
template <int NF, int TPF, bool INV, unsigned MASK>
__device__ __forceinline__ void dif_first_from_regs(float2 *buf, float2 (&v)[16], const float2 *__restrict__ tw,
                                                    int tid) {
    constexpr int ST = NF / 16;
    if (TPF == ST || tid < ST) {
        dft16m<INV, MASK>(v);
        twiddle16<INV>(v, tw + tw_offset<NF, ST>(), ST, tid);
        const int b = dpad(tid);
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[b + r * dpad(ST)] = v[r];   // dpad(tid + r ST) = dpad(tid) + r dpad(ST)
    }
}

// the middle pass (NF = 4096 only: stride 16), ends with a barrier
template <int NF, int TPF, bool INV>
__device__ __forceinline__ void dif_middle(float2 *buf, const float2 *__restrict__ tw, int tid) {
    if constexpr (NF == 4096) {
        constexpr int ST = 16;
        if (TPF == NF / 16 || tid < NF / 16) {
            const int sidx = tid & (ST - 1);
            const int b = dpad((tid >> 4) * 256 + sidx);   // + 17 r for element + 16 r
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = buf[b + 17 * r];
            dft16<INV>(v);
            twiddle16<INV>(v, tw + tw_offset<NF, ST>(), ST, sidx);
#pragma unroll
            for (int r = 0; r < 16; ++r) buf[b + 17 * r] = v[r];
        }
        __syncthreads();
    }
}

// last pass into registers: v[r] = X[tid + r NF/16]; ends with a barrier (SYNC)
template <int NF, int TPF, bool INV, bool SYNC = true>
__device__ __forceinline__ void dif_last_to_regs(const float2 *buf, int tid, float2 (&v)[16]) {
    constexpr int NS = NF / 16;
    if (TPF == NS || tid < NS) {
        const int b = dpad(16 * dif_rev<NF>(tid));   // + r for element + r
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = buf[b + r];
        dft16<INV>(v);
    }
    if constexpr (SYNC) __syncthreads();
}

// ---- The three phases of a frame transform whose input and output are in
// registers, in the in-place form where NF allows it and the Stockham form
// otherwise.  fft_in: first pass (the caller syncs after it); fft_mid: the
// middle passes (each ends with a barrier); fft_out: the last pass.
template <int NF, int TPF, bool INV, unsigned MASK>
__device__ __forceinline__ void fft_in(float2 *buf, float2 (*u)[FftPlan<NF>::R1], const float2 *__restrict__ tw,
                                       int tid) {
    if constexpr (dif_ok<NF>()) dif_first_from_regs<NF, TPF, INV, MASK>(buf, u[0], tw, tid);
    else fft_first_from_regs<NF, TPF, INV, MASK>(buf, u, tid);
}
template <int NF, int TPF, bool INV>
__device__ __forceinline__ void fft_mid(float2 *buf, const float2 *__restrict__ tw, int tid) {
    if constexpr (dif_ok<NF>()) dif_middle<NF, TPF, INV>(buf, tw, tid);
    else fft_middle<NF, TPF, FftPlan<NF>::R1, INV>(buf, tw, tid);
}
template <int NF, int TPF, bool INV, bool SYNC = true>
__device__ __forceinline__ void fft_out(const float2 *buf, const float2 *__restrict__ tw, int tid, float2 (&v)[16]) {
    if constexpr (dif_ok<NF>()) dif_last_to_regs<NF, TPF, INV, SYNC>(buf, tid, v);
    else fft_last_to_regs<NF, TPF, INV, SYNC>(buf, tw, tid, v);
}

// Whole in-place FFT of buf (natural order in and out), for callers that do
// not fuse the first or last pass.  Caller syncs after writing buf; ends with
// a __syncthreads().
template <int NF, int TPF, bool INV>
__device__ __forceinline__ void fft(float2 *buf, const float2 *__restrict__ tw, int tid) {
    constexpr int R1 = FftPlan<NF>::R1;
    stockham_pass<NF, TPF, R1, 1, INV>(buf, tw, tid);
    fft_middle<NF, TPF, R1, INV>(buf, tw, tid);
    stockham_pass<NF, TPF, 16, NF / 16, INV>(buf, tw, tid);
}

}  // namespace sst
