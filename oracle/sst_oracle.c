/*
 * FP64 CPU oracle of the downsampled STFT-based synchrosqueezing transform
 * (He & Cao, "Fast implementation of synchrosqueezing transform based on
 * downsampling for large-scale vibration signal analysis").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant with the CUDA library: it has its own
 * radix-2 FFT, computes every twiddle and phase with libm cos/sin in double,
 * and follows the paper's equations step by step in the paper's order.
 *
 * Conventions (all in samples, not seconds):
 *   window index j runs over [-M, M], M = (L-1)/2, stored at j+M;
 *   frame m is centred on sample m*hop, F = ceil(n/hop) frames, x = 0 outside [0,n);
 *   frequencies are in coarse DFT bins (bin k <-> k*fs/nfft Hz);
 *   complex arrays are interleaved (re, im) doubles.
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   R1 window not renormalised after sampling/truncation;
 *   R2 L > nfft folds the window modulo nfft (time aliasing, Eq. 8 is the definition);
 *   R3 omega_hat kept signed (no modulus), destinations outside the grid dropped as leak;
 *   R4 band [k_lo, k_hi] inclusive; destination l = floor(z*(omega-k_lo) + 1/2);
 *   R5 inverse treats T as the one-sided half of a real frame: factor 2/nfft, weight 1/2 on
 *      the DC and Nyquist destinations, zNf-point IDFT scaled by 1/nfft (not 1/(z nfft));
 *   R6 the 1/sqrt(2) of Eq. 26 is replaced by its exact discrete value, the normaliser
 *      D[p] = g[0] * sum_m g[p - m hop] (the continuous limit of which is sqrt(2)/hop).
 *
 * Parity of every function here is pinned by tests against closed forms, brute
 * force on tiny inputs and invariants; nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORO_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Window tables.  Gaussian g(t) = (pi sigma^2)^(-1/4) exp(-t^2 / (2 sigma^2))   */
/* (Sec. 2.1) and its derivative g'(t) = -(t / sigma^2) g(t) (Sec. 2.2, the      */
/* window of the second STFT), sampled at integer t = j, j in [-M, M].          */
/* ------------------------------------------------------------------------ */
int oro_window(int L, double sigma, double *g, double *dg)
{
    if (L < 1 || (L % 2) == 0 || !(sigma > 0.0)) return -1;
    int M = (L - 1) / 2;
    double amp = pow(ORO_PI * sigma * sigma, -0.25);
    for (int j = -M; j <= M; ++j) {
        double t = (double)j;
        double v = amp * exp(-(t * t) / (2.0 * sigma * sigma));
        g[j + M] = v;
        dg[j + M] = -(t / (sigma * sigma)) * v;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Radix-2 decimation-in-time FFT, in place, unnormalised.                  */
/*   sign = -1: X[k] = sum_n x[n] exp(-2 pi i k n / n_)                      */
/*   sign = +1: x[n] = sum_k X[k] exp(+2 pi i k n / n_)                      */
/* ------------------------------------------------------------------------ */
static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

int oro_fft(double *re, double *im, int64_t n, int sign)
{
    if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    /* butterflies: span len combines two len/2 transforms */
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1;
        double ang = sign * 2.0 * ORO_PI / (double)len;
        for (int64_t q = 0; q < half; ++q) {
            double wr = cos(ang * (double)q), wi = sin(ang * (double)q);
            for (int64_t s = q; s < n; s += len) {
                int64_t t = s + half;
                double br = re[t] * wr - im[t] * wi;
                double bi = re[t] * wi + im[t] * wr;
                re[t] = re[s] - br; im[t] = im[s] - bi;
                re[s] += br;        im[s] += bi;
            }
        }
    }
    return 0;
}

/* Plain O(n^2) DFT with the same sign convention, for sizes that are not a
 * power of two (the zNf-point inverse when z is not a power of two). */
static void dft_direct(double *re, double *im, int64_t n, int sign)
{
    double *or_ = (double *)malloc(sizeof(double) * (size_t)n);
    double *oi = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t t = 0; t < n; ++t) {
            double a = sign * 2.0 * ORO_PI * (double)((k * t) % n) / (double)n;
            double c = cos(a), s = sin(a);
            sr += re[t] * c - im[t] * s;
            si += re[t] * s + im[t] * c;
        }
        or_[k] = sr; oi[k] = si;
    }
    memcpy(re, or_, sizeof(double) * (size_t)n);
    memcpy(im, oi, sizeof(double) * (size_t)n);
    free(or_); free(oi);
}

static void transform(double *re, double *im, int64_t n, int sign)
{
    if (is_pow2(n)) oro_fft(re, im, n, sign);
    else dft_direct(re, im, n, sign);
}

int64_t oro_frames(int64_t n, int hop) { return (n + hop - 1) / hop; }

/* ------------------------------------------------------------------------ */
/* Downsampled STFT, Eq. 9:                                                  */
/*   S[m,k] = exp(i 2 pi k M / Nf) sum_{t=0}^{Nf-1} x[t + m hop - M] g[t - M]  */
/*            exp(-i 2 pi k t / Nf)                                          */
/* for frames m in [m0, m0+nm) and bins k in [k_lo, k_hi].  The summand runs */
/* over the window support t in [0, L); for L > Nf the index is folded mod   */
/* Nf (reading R2: Eq. 8 is the definition, and its DFT samples fold).       */
/* Computes S with window g into V and with window g' into Vd.               */
/* ------------------------------------------------------------------------ */
int oro_stft(const double *x, int64_t n, const double *g, const double *dg,
             int L, int hop, int nfft, int64_t m0, int64_t nm,
             int k_lo, int k_hi, double *V, double *Vd)
{
    if (!is_pow2(nfft) || L < 1 || (L % 2) == 0 || hop < 1) return -1;
    if (k_lo < 0 || k_hi > nfft / 2 || k_lo > k_hi) return -1;
    int M = (L - 1) / 2;
    int nb = k_hi - k_lo + 1;
    int err = 0;
#pragma omp parallel
    {
        double *re = (double *)malloc(sizeof(double) * (size_t)nfft);
        double *im = (double *)malloc(sizeof(double) * (size_t)nfft);
        if (!re || !im) err = -2;
#pragma omp for schedule(static)
        for (int64_t mi = 0; mi < nm; ++mi) {
            if (!re || !im) continue;
            int64_t m = m0 + mi;
            for (int w = 0; w < 2; ++w) {
                const double *win = (w == 0) ? g : dg;
                double *out = (w == 0) ? V : Vd;
                memset(re, 0, sizeof(double) * (size_t)nfft);
                memset(im, 0, sizeof(double) * (size_t)nfft);
                for (int t = 0; t < L; ++t) {
                    int64_t s = m * (int64_t)hop - M + t;
                    double xs = (s >= 0 && s < n) ? x[s] : 0.0;
                    re[t % nfft] += xs * win[t];
                }
                oro_fft(re, im, nfft, -1);
                for (int k = k_lo; k <= k_hi; ++k) {
                    double a = 2.0 * ORO_PI * (double)(((int64_t)k * M) % nfft) / (double)nfft;
                    double c = cos(a), s = sin(a);
                    double *o = out + 2 * ((size_t)mi * nb + (k - k_lo));
                    o[0] = c * re[k] - s * im[k];
                    o[1] = c * im[k] + s * re[k];
                }
            }
        }
        free(re); free(im);
    }
    return err;
}

/* ------------------------------------------------------------------------ */
/* Instantaneous-frequency estimate and selective, subdivided reassignment.  */
/*   Eq. 12-13 / Eq. 36: omega[m,k] = k - (Nf / 2 pi) Im(Vd[m,k] / V[m,k])    */
/*   (in coarse bins; signed, reading R3), computed where V != 0.            */
/*   Threshold |V| > gamma (Eq. 13).                                        */
/*   Eq. 27-29: grid xi*[l] = k_lo + l / z, l = 0 .. z N_r, N_r = k_hi-k_lo, */
/*   and |omega - xi*[l]| <= 1/(2z) picks l = floor(z (omega - k_lo) + 1/2)  */
/*   (reading R4: a single destination, ties go up).                          */
/*   T[m,l] = sum over source bins k (ascending) with destination l of V.     */
/*   Destinations outside [0, z N_r] are accumulated into leak[m].           */
/* dest[m,k] = l, or -1 below threshold, or -2 outside the grid.             */
/* ------------------------------------------------------------------------ */
int oro_reassign(const double *V, const double *Vd, int64_t nm, int k_lo, int k_hi,
                 int nfft, int z, double gamma,
                 double *omega, int32_t *dest, double *T, double *leak)
{
    if (z < 1 || k_lo > k_hi) return -1;
    int nb = k_hi - k_lo + 1;
    int nbo = z * (k_hi - k_lo) + 1;
    double c = (double)nfft / (2.0 * ORO_PI);
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < nm; ++m) {
        double *Trow = T ? T + 2 * (size_t)m * nbo : NULL;
        if (Trow) memset(Trow, 0, sizeof(double) * 2 * (size_t)nbo);
        double lr = 0.0, li = 0.0;
        for (int k = k_lo; k <= k_hi; ++k) {
            size_t i = (size_t)m * nb + (k - k_lo);
            double vr = V[2 * i], vi = V[2 * i + 1];
            double dr = Vd[2 * i], di = Vd[2 * i + 1];
            double mag2 = vr * vr + vi * vi;
            double om = NAN;
            if (mag2 > 0.0) {
                double im_ratio = (di * vr - dr * vi) / mag2;   /* Im(Vd / V) */
                om = (double)k - c * im_ratio;
            }
            if (omega) omega[i] = om;
            if (!(hypot(vr, vi) > gamma)) {   /* |V| > gamma, Eq. 13 */
                if (dest) dest[i] = -1;
                continue;
            }
            double u = (double)z * (om - (double)k_lo);
            double lf = floor(u + 0.5);
            if (!(lf >= 0.0 && lf <= (double)(nbo - 1))) {
                if (dest) dest[i] = -2;
                lr += vr; li += vi;
                continue;
            }
            int l = (int)lf;
            if (dest) dest[i] = l;
            if (Trow) { Trow[2 * l] += vr; Trow[2 * l + 1] += vi; }
        }
        if (leak) { leak[2 * m] = lr; leak[2 * m + 1] = li; }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Inverse normaliser of reading R6, Eq. 26:                                */
/*   D[p] = g[0] * sum_{m=0}^{F-1} g[p - m hop]        (mode 0, Eq. 26)       */
/* and the WOLA normaliser of Eq. 11:                                        */
/*   D[p] = sum_{m=0}^{F-1} g[p - m hop]^2              (mode 1, Eq. 10-11)   */
/* g is zero outside [-M, M].                                                */
/* ------------------------------------------------------------------------ */
static double normaliser(const double *g, int L, int hop, int64_t F, int64_t p, int mode)
{
    int M = (L - 1) / 2;
    /* frames whose support [m hop - M, m hop + M] contains p */
    int64_t mlo = (p - M > 0) ? (p - M + hop - 1) / hop : 0;
    int64_t mhi = (p + M) / hop;
    if (mhi > F - 1) mhi = F - 1;
    double s = 0.0;
    for (int64_t m = mlo; m <= mhi; ++m) {
        int64_t j = p - m * hop;
        if (j < -M || j > M) continue;
        double w = g[j + M];
        s += (mode == 0) ? w : w * w;
    }
    return (mode == 0) ? g[M] * s : s;
}

int oro_normaliser(const double *g, int L, int hop, int64_t F, int64_t p0, int64_t np,
                   int mode, double *D)
{
    for (int64_t i = 0; i < np; ++i) D[i] = normaliser(g, L, hop, F, p0 + i, mode);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Direct approximate inverse, Eq. 25-26 with P. 223's zero padding:          */
/*   spectrum on the z Nf grid: bin kk = z k_lo + l holds                     */
/*        w_kk * T[m,l] * exp(-i 2 pi kk M / (z Nf)),                         */
/*        w = 1/2 at DC (kk = 0) and Nyquist (kk = z Nf / 2), else 1 (R5);     */
/*   zNf-point inverse DFT, real part, times 2/Nf (R5):  r~[m,t], t in [0,L)  */
/*   (index t taken mod zNf), at time m hop - M + t;                          */
/*   overlap-add  num[p] = sum_m g[t] r~[m,t],  xhat[p] = num[p] / D[p] (R6).  */
/* Output samples p in [p0, p0+np).  T holds frames [mt0, mt0+ntf), which     */
/* must cover every frame that touches the output range.                     */
/* mode 0 = Eq. 26 normaliser, mode 1 = Eq. 11 WOLA normaliser (Sum g^2),     */
/* mode 2 = the overlap-add numerator of the frames T holds alone, not divided */
/* (the share of one contiguous range of frames, for a signal split by frame */
/* ranges; T then need not cover every frame touching the output range).     */
/* ------------------------------------------------------------------------ */
/* r~[m, t] for t in [0, L) of one frame (Eq. 25 on the zero-padded z Nf grid),
 * from its T row; re, im are G = z Nf doubles of scratch. */
static void frame_rtilde(const double *Trow, int k_lo, int nbo, int nfft, int z, int L, int M,
                         double *re, double *im, double *rt)
{
    int64_t G = (int64_t)z * nfft;
    memset(re, 0, sizeof(double) * (size_t)G);
    memset(im, 0, sizeof(double) * (size_t)G);
    for (int l = 0; l < nbo; ++l) {
        int64_t kk = (int64_t)z * k_lo + l;
        double w = (kk == 0 || 2 * kk == G) ? 0.5 : 1.0;
        double a = -2.0 * ORO_PI * (double)((kk * M) % G) / (double)G;
        double c = cos(a), s = sin(a);
        double tr = Trow[2 * l], ti = Trow[2 * l + 1];
        re[kk] += w * (tr * c - ti * s);
        im[kk] += w * (tr * s + ti * c);
    }
    transform(re, im, G, +1);
    for (int t = 0; t < L; ++t) rt[t] = (2.0 / (double)nfft) * re[t % G];
}

int oro_inverse(const double *T, int64_t mt0, int64_t ntf, int k_lo, int nbo, int nfft, int z,
                const double *g, int L, int hop, int64_t n, int64_t p0, int64_t np,
                int mode, double *xhat)
{
    if (z < 1 || L < 1 || (L % 2) == 0 || hop < 1 || np < 0) return -1;
    int M = (L - 1) / 2;
    int64_t F = oro_frames(n, hop);
    int64_t G = (int64_t)z * nfft;
    if ((int64_t)z * k_lo + nbo - 1 > G / 2) return -1;
    if (np == 0) return 0;
    int64_t pend = p0 + np - 1;
    int64_t mlo = (p0 - M > 0) ? (p0 - M + hop - 1) / hop : 0;
    int64_t mhi = (pend + M) / hop;
    if (mhi > F - 1) mhi = F - 1;
    if (mode == 2) {                                   /* the given frames only */
        if (mlo < mt0) mlo = mt0;
        if (mhi > mt0 + ntf - 1) mhi = mt0 + ntf - 1;
    } else if (mlo < mt0 || mhi > mt0 + ntf - 1) {
        return -3;                                     /* T does not cover the range */
    }

    /* Frames are taken in chunks: the r~ of a chunk's frames are independent
     * (Eq. 25) and computed in parallel; they are then overlap-added one frame
     * after another in ascending frame order (Eq. 26), so every output sample
     * sums its frames in the same order for any number of threads. */
    const int64_t chunk = 256;
    double *num = (double *)calloc((size_t)np, sizeof(double));
    double *seg = (double *)malloc(sizeof(double) * (size_t)chunk * (size_t)L);
    if (!num || !seg) { free(num); free(seg); return -2; }
    int failed = 0;
    for (int64_t c0 = mlo; c0 <= mhi && !failed; c0 += chunk) {
        int64_t cn = (mhi - c0 + 1 < chunk) ? mhi - c0 + 1 : chunk;
#pragma omp parallel
        {
            double *re = (double *)malloc(sizeof(double) * (size_t)G);
            double *im = (double *)malloc(sizeof(double) * (size_t)G);
            if (!re || !im) {
#pragma omp atomic write
                failed = 1;
            }
#pragma omp for schedule(static)
            for (int64_t i = 0; i < cn; ++i)
                if (re && im)
                    frame_rtilde(T + 2 * (size_t)(c0 + i - mt0) * nbo, k_lo, nbo, nfft, z, L, M, re, im,
                                 seg + (size_t)i * L);
            free(re);
            free(im);
        }
        if (failed) break;
        for (int64_t i = 0; i < cn; ++i) {
            int64_t m = c0 + i;
            for (int t = 0; t < L; ++t) {
                int64_t p = m * (int64_t)hop - M + t;
                if (p < p0 || p > pend) continue;
                num[p - p0] += g[t] * seg[(size_t)i * L + t];
            }
        }
    }
    if (failed) { free(num); free(seg); return -2; }
    for (int64_t i = 0; i < np; ++i)
        xhat[i] = (mode == 2) ? num[i] : num[i] / normaliser(g, L, hop, F, p0 + i, mode);
    free(num); free(seg);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Standard (full-sampled) inverse, Eq. 15 with the whole grid as the zone:  */
/*   x[m] = 1/(2 pi g(0)) Re( sum over the two-sided grid of T d xi ),       */
/* d xi = 2 pi / Nf per coarse bin; with the one-sided T of reading R5 this  */
/*   x[m] = (2 / (Nf g(0))) Re sum_l w_l T[m,l].                              */
/* Valid for hop = 1, where frame m sits at sample m.  With subdivision the  */
/* coefficients are moved to finer bins, not split, so no 1/z appears; z     */
/* only locates the DC and Nyquist destinations.                             */
/* ------------------------------------------------------------------------ */
int oro_colsum(const double *T, int64_t nm, int k_lo, int nbo, int nfft, int z, double g0,
               double *xcol)
{
    int64_t G = (int64_t)z * nfft;
    for (int64_t m = 0; m < nm; ++m) {
        double s = 0.0;
        for (int l = 0; l < nbo; ++l) {
            int64_t kk = (int64_t)z * k_lo + l;
            double w = (kk == 0 || 2 * kk == G) ? 0.5 : 1.0;
            s += w * T[2 * ((size_t)m * nbo + l)];
        }
        xcol[m] = 2.0 * s / ((double)nfft * g0);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Parameter relations of Sec. 4 (sigma in seconds, fs in Hz):               */
/*   Eq. 35  sigma_f = 1 / (2 pi sigma)                                      */
/*   Eq. 38  Hf < 3 N / (4 pi sigma fs)                                      */
/*   Eq. 46  Delta f < sqrt(2) sigma_f, i.e. Hf < sqrt(2) sigma_f N / fs     */
/*   Eq. 12 / 28  Delta f = fs / Nf, subdivided Delta f* = fs / (z Nf)        */
/* ------------------------------------------------------------------------ */
/* Threads the OpenMP loops above may use (timing only; results do not depend on it). */
#ifdef _OPENMP
#include <omp.h>
void oro_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }
int oro_get_threads(void) { return omp_get_max_threads(); }
#else
void oro_set_threads(int n) { (void)n; }
int oro_get_threads(void) { return 1; }
#endif

double oro_sigma_f(double sigma_s) { return 1.0 / (2.0 * ORO_PI * sigma_s); }
double oro_hf_max_rule1(double n, double sigma_s, double fs) { return 3.0 * n / (4.0 * ORO_PI * sigma_s * fs); }
double oro_hf_max_rule2(double n, double sigma_s, double fs) { return sqrt(2.0) * oro_sigma_f(sigma_s) * n / fs; }
double oro_delta_f(double fs, int nfft, int z) { return fs / ((double)nfft * (double)z); }
