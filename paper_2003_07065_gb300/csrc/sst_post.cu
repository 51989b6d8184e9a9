// Steps after the transform: ridge extraction on T (the ridges that Sec. 2.2
// builds the Eq. 15 zone around and Sec. 5 tracks) and the Renyi entropy of
// Eq. 32 (the concentration measure of Sec. 3.2).  Both stream T from HBM:
// the ridge once, the entropy twice (its exact maximum, then its sums).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "sst_internal.h"

namespace sst {
namespace {

// ---------------------------------------------------------------- ridge
// One CTA per tile of RIDGE_TB frames (grid-stride).  Thread t owns output
// bin l = c0 + t of each 256-bin chunk c0 of the band: it stages |T|^2 of
// the tile's frames and the smooth frames on either side in its own column
// of shared memory, forms E[m, l] for every frame of the tile (d ascending)
// and keeps, per frame, its largest E (the earlier chunk, i.e. the smaller
// l, on equality).  A per-frame reduction over the CTA then picks the
// largest E and the smallest l among equals.  A thread touches only its own
// column, so staging needs no barrier.
constexpr int RIDGE_THREADS = 256;
constexpr int RIDGE_TB = 16;

__device__ __forceinline__ bool ridge_better(float e, int l, float e2, int l2) {
    return e > e2 || (e == e2 && (unsigned)l < (unsigned)l2);   // l = -1 (none) loses ties
}

__global__ void __launch_bounds__(RIDGE_THREADS, 4)
k_ridge(const float2 *__restrict__ T, int64_t F, int ld, int l_lo, int l_hi, int smooth, int32_t *__restrict__ ridge) {
    extern __shared__ float P[];   // (RIDGE_TB + 2 smooth) rows x RIDGE_THREADS columns
    __shared__ float wE[RIDGE_TB][RIDGE_THREADS / 32];
    __shared__ int wL[RIDGE_TB][RIDGE_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rows = RIDGE_TB + 2 * smooth;
    const int64_t tiles = (F + RIDGE_TB - 1) / RIDGE_TB;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t m0 = tile * RIDGE_TB;
        float bE[RIDGE_TB];
        int bL[RIDGE_TB];
#pragma unroll
        for (int i = 0; i < RIDGE_TB; ++i) {
            bE[i] = -1.f;
            bL[i] = -1;
        }
        for (int c0 = l_lo; c0 <= l_hi; c0 += RIDGE_THREADS) {
            const int l = c0 + tid;
            if (l > l_hi) break;
            // eight independent (predicated) loads in flight per batch
            for (int r0 = 0; r0 < rows; r0 += 8) {
                float2 t[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t m = m0 - smooth + r0 + u;
                    t[u] = (r0 + u < rows && m >= 0 && m < F) ? T[m * ld + l] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (r0 + u < rows) P[(r0 + u) * RIDGE_THREADS + tid] = t[u].x * t[u].x + t[u].y * t[u].y;
            }
#pragma unroll
            for (int i = 0; i < RIDGE_TB; ++i) {
                float e = 0.f;
                for (int d = 0; d <= 2 * smooth; ++d) e += P[(i + d) * RIDGE_THREADS + tid];
                if (e > bE[i]) {
                    bE[i] = e;
                    bL[i] = l;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RIDGE_TB; ++i) {
            float e = bE[i];
            int l = bL[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
                const int l2 = __shfl_xor_sync(0xffffffffu, l, o);
                if (ridge_better(e2, l2, e, l)) {
                    e = e2;
                    l = l2;
                }
            }
            if (lane == 0) {
                wE[i][warp] = e;
                wL[i][warp] = l;
            }
        }
        __syncthreads();
        if (tid < RIDGE_TB && m0 + tid < F) {
            float e = wE[tid][0];
            int l = wL[tid][0];
            for (int w = 1; w < RIDGE_THREADS / 32; ++w)
                if (ridge_better(wE[tid][w], wL[tid][w], e, l)) {
                    e = wE[tid][w];
                    l = wL[tid][w];
                }
            ridge[m0 + tid] = (e > 0.f) ? l : -1;
        }
        __syncthreads();   // wE, wL are rewritten by the next tile
    }
}

// ---------------------------------------------------------------- Renyi
// Two passes over the grid.  The first finds M = max P exactly (atomicMax on
// the bits of non-negative floats, order independent).  The second sums
// q = P/M <= 1 and q^alpha: a thread's terms of four rows in FP32, then
// folded into FP64, the threads of a block combined in a fixed tree
// order and the blocks by one final block, so the result does not depend on
// scheduling.  Only additions touch FP64 (slow on this part).
constexpr int RENYI_THREADS = 256;
constexpr int RENYI_MAX_BLOCKS = 1024;
struct RenyiPart {
    double s1, sa;
};

__device__ __forceinline__ float pow_alpha(float q, float alpha, int ai) {
    if (ai == 2) return q * q;
    if (ai == 3) return q * q * q;
    return q > 0.f ? exp2f(alpha * log2f(q)) : 0.f;
}

// A thread's share of one row, eight columns RENYI_THREADS apart per batch,
// the loads of a batch issued together.
template <typename F>
__device__ __forceinline__ void renyi_row(const float2 *__restrict__ row, int cols, int tid, F &&f) {
    for (int c0 = 0; c0 < cols; c0 += 8 * RENYI_THREADS) {
        float2 t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + u * RENYI_THREADS + tid;
            t[u] = c < cols ? row[c] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) f(t[u].x * t[u].x + t[u].y * t[u].y);
    }
}

__global__ void __launch_bounds__(RENYI_THREADS)
k_renyi_max(const float2 *__restrict__ T, int64_t rows, int cols, int64_t ld, unsigned *__restrict__ mbits) {
    __shared__ float red[RENYI_THREADS / 32];
    const int tid = threadIdx.x;
    float m = 0.f;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
        renyi_row(T + r * ld, cols, tid, [&](float p) { m = fmaxf(m, p); });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < RENYI_THREADS / 32; ++w) m = fmaxf(m, red[w]);
        if (m > 0.f) atomicMax(mbits, __float_as_uint(m));
    }
}

__global__ void __launch_bounds__(RENYI_THREADS)
k_renyi_partial(const float2 *__restrict__ T, int64_t rows, int cols, int64_t ld, float alpha, int ai,
                const unsigned *__restrict__ mbits, RenyiPart *__restrict__ part) {
    __shared__ double s1s[RENYI_THREADS], sas[RENYI_THREADS];
    const int tid = threadIdx.x;
    const float M = __uint_as_float(*mbits);
    const float rM = M > 0.f ? 1.f / M : 0.f;
    float c1 = 0.f, ca = 0.f;
    double s1 = 0.0, sa = 0.0;
    int k = 0;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        renyi_row(T + r * ld, cols, tid, [&](float p) {
            const float q = fminf(p * rM, 1.f);
            c1 += q;
            ca += pow_alpha(q, alpha, ai);
        });
        // fold every 4 rows: at most 4 ceil(cols / RENYI_THREADS) FP32 terms, each <= 1
        if (++k == 4) {
            s1 += c1;
            sa += ca;
            c1 = ca = 0.f;
            k = 0;
        }
    }
    s1s[tid] = s1 + c1;
    sas[tid] = sa + ca;
    __syncthreads();
    for (int o = RENYI_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) {
            s1s[tid] += s1s[tid + o];
            sas[tid] += sas[tid + o];
        }
        __syncthreads();
    }
    if (tid == 0) part[blockIdx.x] = RenyiPart{s1s[0], sas[0]};
}

__global__ void __launch_bounds__(RENYI_THREADS)
k_renyi_final(const RenyiPart *__restrict__ part, int nparts, const unsigned *__restrict__ mbits, double alpha,
              double cell, double *__restrict__ out) {
    __shared__ double s1s[RENYI_THREADS], sas[RENYI_THREADS];
    const int tid = threadIdx.x;
    double s1 = 0.0, sa = 0.0;
    for (int i = tid; i < nparts; i += RENYI_THREADS) {
        s1 += part[i].s1;
        sa += part[i].sa;
    }
    s1s[tid] = s1;
    sas[tid] = sa;
    __syncthreads();
    for (int o = RENYI_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) {
            s1s[tid] += s1s[tid + o];
            sas[tid] += sas[tid + o];
        }
        __syncthreads();
    }
    // sum (P / sum P)^alpha = (M^alpha Sa) / (M S1)^alpha = Sa / S1^alpha
    if (tid == 0)
        *out = (*mbits != 0u) ? (log2(sas[0]) - alpha * log2(s1s[0])) / (1.0 - alpha) + log2(cell) : nan("");
}

std::once_flag g_ridge_attr;
cudaError_t g_ridge_attr_err = cudaSuccess;

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

}  // namespace
}  // namespace sst

using namespace sst;

SST_API sst_status sst_ridge(const float *tfr_dev, int64_t frames, int32_t bins, int32_t l_lo, int32_t l_hi,
                             int32_t smooth, int32_t *ridge_dev, void *stream) {
    SST_NVTX_RANGE();
    if (!tfr_dev || !ridge_dev) return fail(SST_EINVAL, "tfr or ridge pointer is NULL");
    if (((uintptr_t)tfr_dev) & 7) return fail(SST_EINVAL, "tfr must be 8-byte aligned");
    if (((uintptr_t)ridge_dev) & 3) return fail(SST_EINVAL, "ridge must be 4-byte aligned");
    if (frames < 1 || bins < 1) return fail(SST_EINVAL, "empty TFR (%lld x %d)", (long long)frames, bins);
    if (l_lo < 0 || l_hi < l_lo || l_hi >= bins)
        return fail(SST_EINVAL, "band [%d, %d] outside [0, %d)", l_lo, l_hi, bins);
    if (smooth < 0 || smooth > SST_RIDGE_MAX_SMOOTH)
        return fail(SST_EINVAL, "smooth = %d outside [0, %d]", smooth, SST_RIDGE_MAX_SMOOTH);
    std::call_once(g_ridge_attr, [] {
        g_ridge_attr_err = cudaFuncSetAttribute(k_ridge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)(sizeof(float) * RIDGE_THREADS *
                                                      (RIDGE_TB + 2 * SST_RIDGE_MAX_SMOOTH)));
    });
    SST_CU(g_ridge_attr_err, "cudaFuncSetAttribute");
    const int sms = device_sms();
    if (sms < 1) return fail(SST_ECUDA, "no device");
    const int64_t tiles = (frames + RIDGE_TB - 1) / RIDGE_TB;
    const size_t smem = sizeof(float) * RIDGE_THREADS * (RIDGE_TB + 2 * (size_t)smooth);
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ridge, RIDGE_THREADS, smem) != cudaSuccess || occ < 1)
        occ = 1;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)occ * sms);
    cudaStream_t st = (cudaStream_t)stream;
    SST_LAUNCHED_K(PK_OTHER, st,
                   (k_ridge<<<(unsigned)grid, RIDGE_THREADS, smem, st>>>((const float2 *)tfr_dev, frames, bins, l_lo,
                                                                          l_hi, smooth, ridge_dev),
                    cudaGetLastError()),
                   "ridge launch");
    return SST_OK;
}

// workspace: the max word (256 bytes reserved), then the block partials
SST_API size_t sst_renyi_workspace_bytes(void) { return 256 + sizeof(RenyiPart) * RENYI_MAX_BLOCKS; }

SST_API sst_status sst_renyi(const float *tfr_dev, int64_t rows, int32_t cols, int64_t ld, double alpha, double cell,
                             double *out_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    if (!tfr_dev || !out_dev || !ws) return fail(SST_EINVAL, "tfr, out or workspace pointer is NULL");
    if (((uintptr_t)tfr_dev) & 7) return fail(SST_EINVAL, "tfr must be 8-byte aligned");
    if (((uintptr_t)out_dev) & 7) return fail(SST_EINVAL, "out must be 8-byte aligned");
    if (((uintptr_t)ws) & 255) return fail(SST_EINVAL, "workspace must be 256-byte aligned");
    if (rows < 1 || cols < 1 || ld < cols) return fail(SST_EINVAL, "bad grid %lld x %d (ld %lld)", (long long)rows, cols,
                                                    (long long)ld);
    if (!(alpha > 0.0) || alpha == 1.0 || !std::isfinite(alpha)) return fail(SST_EINVAL, "alpha must be > 0 and != 1");
    if (!(cell > 0.0) || !std::isfinite(cell)) return fail(SST_EINVAL, "cell must be > 0");
    const int sms = device_sms();
    if (sms < 1) return fail(SST_ECUDA, "no device");
    const int grid = (int)std::min<int64_t>(rows, std::min<int64_t>(RENYI_MAX_BLOCKS, 8LL * sms));
    const int ai = alpha == 2.0 ? 2 : (alpha == 3.0 ? 3 : 0);
    unsigned *mbits = (unsigned *)ws;
    RenyiPart *part = (RenyiPart *)((char *)ws + 256);
    cudaStream_t st = (cudaStream_t)stream;
    const float2 *T = (const float2 *)tfr_dev;
    SST_CU(cudaMemsetAsync(mbits, 0, sizeof(unsigned), st), "renyi memset");
    SST_LAUNCHED_K(PK_OTHER, st,
                   (k_renyi_max<<<grid, RENYI_THREADS, 0, st>>>(T, rows, cols, ld, mbits), cudaGetLastError()),
                   "renyi max launch");
    SST_LAUNCHED_K(PK_OTHER, st,
                   (k_renyi_partial<<<grid, RENYI_THREADS, 0, st>>>(T, rows, cols, ld, (float)alpha, ai, mbits, part),
                    cudaGetLastError()),
                   "renyi launch");
    SST_LAUNCHED_K(PK_OTHER, st,
                   (k_renyi_final<<<1, RENYI_THREADS, 0, st>>>(part, grid, mbits, alpha, cell, out_dev),
                    cudaGetLastError()),
                   "renyi final launch");
    return SST_OK;
}
