// Band-limited tensor-core form of the STFT pair (the precision study of the
// in-band bins): for frames m and band bins k,
//   [Re V, Im V, Re V', Im V'][m, k] = sum_j x[m hop + j - M] B[j, 4k + c]
// with B[j, .] = (g cos, -g sin, s g' cos, -s g' sin)(2 pi k (j - M) / Nf)
// (Eq. 8, the direct sum, so L > Nf needs no folding), computed as a
// [frames x L] x [L x 4 nb] contraction on tcgen05 with FP32 accumulation in
// tensor memory.  Operands: plain BF16, BF16 split hi + lo (three products
// hi.hi + hi.lo + lo.hi), or TF32.  A is the Hankel view of the zero-padded
// signal (rows H samples apart) when the tensor-map encoder accepts
// overlapping rows, else an explicit frames x L copy.  The same IF /
// threshold / reassignment epilogue as the FFT form then produces T.
//
// GEMM kernel: one CTA per 128 x 256 output tile; warp 0 issues TMA loads into
// a 4-stage shared-memory ring, one thread of warp 1 issues tcgen05.mma
// (M 128, N 256, 32 bytes of K per instruction), warps 2-5 read the
// accumulator back with tcgen05.ld.  Every mbarrier wait is bounded (about a
// second of clock cycles); on expiry the kernel records the site in an error
// word, drains its own copies in flight (bounded again), frees tensor memory
// and returns, and the host reports SST_ETIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "sst_internal.h"
#include "sst_tc.h"
#include "sst_async.cuh"
#include "sst_kernels.cuh"

namespace sst {
namespace tc {

constexpr int BM = 128, BN = 256;
constexpr int KB = 128;                      // bytes of K per stage (64 bf16 or 32 fp32)
constexpr int STAGES = 4;
constexpr int A_TILE = BM * KB;              // 16 KB
constexpr int B_TILE = BN * KB;              // 32 KB
constexpr int STAGE = A_TILE + B_TILE;
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 256;
constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(su32(dst)),
        "l"((uint64_t)map), "r"(su32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// K-major operand, 128-byte swizzle: 8-row atoms of 128-byte rows, 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset between 8-row atoms
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N = 256
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (TF32)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
            "l"(a), "l"(b), "r"(idesc(2)), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
            "l"(a), "l"(b), "r"(idesc(1)), "r"(acc));
}
// the same load delivered to the same offset (data and barrier) in every CTA
// of the cluster named in mask
__device__ __forceinline__ void tma_2d_mc(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                          uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%3, "
        "%4}], [%2], %5;" ::"r"(su32(dst)),
        "l"((uint64_t)map), "r"(su32(bar)), "r"(c0), "r"(c1), "h"(mask)
        : "memory");
}
// arrive on the barrier at this offset in every CTA of mask once the products issued so far complete
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            su32(bar)),
        "h"(mask)
        : "memory");
}
// one 32-byte store (whole sectors) of 8 floats
__device__ __forceinline__ void st_v8(float *p, const float *v) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// ---- CTA pairs (tcgen05 cta_group::2): one MMA of M = 256 rows across two SMs
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
// load into this CTA's shared memory, completion counted on a barrier that
// may live in the peer CTA (cluster address)
__device__ __forceinline__ void tma_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cluster, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(su32(dst)),
        "l"((uint64_t)map), "r"(bar_cluster), "r"(c0), "r"(c1)
        : "memory");
}
template <bool TF32>
__device__ __forceinline__ void mma_pair(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (TF32)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
            "l"(a), "l"(b), "r"(id), "r"(acc));
}
// arrive on the barrier at this offset in both CTAs of the pair once the pair's products issued so far complete
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            su32(bar)),
        "h"((uint16_t)3)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}
__device__ __forceinline__ bool mbar_try_acq_cluster(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *b, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_acq_cluster(b, parity))
        if (clock64() - t0 > WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// C[rows x ldc] (FP32) = sum over `passes` products of A_p [rows x K] and B_p^T:
// pass 0 A0.B0, pass 1 A0.B1, pass 2 A1.B0 (the BF16 hi / lo split).
// Persistent: CTA b takes tiles b, b + grid, ... (row blocks fastest, so the
// CTAs running together share the basis columns they read); the
// accumulator is double-buffered in tensor memory so the read-back of one
// tile overlaps the products of the next.  The epilogue also folds
// max |S^g|^2 over the valid rows and the first vcols columns into *maxbits
// (the bits of a non-negative float, which order like the floats).
// With CL > 1 the CTAs of a cluster take CL consecutive row blocks of the
// same column block: each loads 1/CL of the basis tile and multicasts it to
// all, so every CTA reads its A tile plus 1/CL of the B tile from L2 per
// stage; a stage is refilled only when every CTA of the cluster is done
// with it.
template <bool TF32, int CL>
__global__ void __launch_bounds__(THREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
          const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1, float *__restrict__ C,
          int rows, int ldc, int vcols, int mtiles, int ntiles, int ktiles, int passes,
          unsigned *__restrict__ maxbits, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;    // accumulator buffer b holds a finished tile
    uint64_t *tempty = tfull + 2;        // accumulator buffer b has been read back
    uint64_t *drain = tempty + 2;        // every product issued has completed
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *issued_s = (volatile int *)(tmem_slot + 1);
    volatile int *consumed_s = issued_s + 1;
    volatile int *failed_s = issued_s + 2;
    const bool withhold = err[1] != 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // cluster c of CL CTAs takes super tiles c, c + clusters, ...: CL row
    // blocks x one column block, row block CL i + rank for this CTA
    const int rank = (CL > 1) ? (int)cluster_rank() : 0;
    const int cid = blockIdx.x / CL, clusters = gridDim.x / CL;
    const int mgroups = mtiles / CL;
    const int tiles = mgroups * ntiles;
    const int per_tile = ktiles * passes;
    constexpr int KEL = TF32 ? 32 : 64;   // K elements per stage

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], CL);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(drain, 1);
        *issued_s = 0;
        *consumed_s = 0;
        *failed_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(2 * TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    if (CL > 1) cluster_sync();   // peers' barriers are initialised before any multicast reaches them
    fence_after();
    const uint32_t tbase = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: one global stage counter over all tiles of this CTA
        int it = 0;
        bool ok = true;
        for (int t = cid; t < tiles && ok; t += clusters) {
            const int m0 = ((t % mgroups) * CL + rank) * BM, n0 = (t / mgroups) * BN;
            for (int j = 0; j < per_tile; ++j, ++it) {
                const int s = it % STAGES;
                if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1)) {
                    atomicOr(err, 1);
                    *failed_s = 1;
                    ok = false;
                    break;
                }
                const int pass = j / ktiles, kt = j % ktiles;
                const CUtensorMap *ma = (pass == 2) ? &tmA1 : &tmA0;
                const CUtensorMap *mb = (pass == 1) ? &tmB1 : &tmB0;
                uint8_t *sa = smem + s * STAGE, *sb = sa + A_TILE;
                // test hook (err[1] != 0): CTA 0 withholds its first stage, so the
                // product's bounded waits run out and report, with no fault
                if (it == 0 && blockIdx.x == 0 && withhold) continue;
                mbar_expect_tx(&full[s], STAGE);
                tma_2d(sa, ma, &full[s], kt * KEL, m0);
                if (CL == 1)
                    tma_2d(sb, mb, &full[s], kt * KEL, n0);
                else
                    tma_2d_mc(sb + rank * (B_TILE / CL), mb, &full[s], kt * KEL, n0 + rank * (BN / CL),
                              (uint16_t)((1u << CL) - 1));
            }
        }
        *issued_s = it;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        int it = 0, lt = 0;
        bool ok = true;
        for (int t = cid; t < tiles && ok; t += clusters, ++lt) {
            const int b = lt & 1;
            if (lt >= 2 && !mbar_wait(&tempty[b], ((lt >> 1) & 1) ^ 1)) {
                atomicOr(err, 2);
                *failed_s = 1;
                break;
            }
            fence_after();
            const uint32_t dt = tbase + (uint32_t)(b * TMEM_COLS);
            for (int j = 0; j < per_tile; ++j, ++it) {
                const int s = it % STAGES;
                if (!mbar_wait(&full[s], (it / STAGES) & 1)) {
                    atomicOr(err, 4);
                    *failed_s = 1;
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t sa = su32(smem + s * STAGE), sb = sa + A_TILE;
#pragma unroll
                for (int k = 0; k < KB / 32; ++k)
                    mma<TF32>(dt, sdesc(sa + 32 * k), sdesc(sb + 32 * k), (j > 0 || k > 0) ? 1u : 0u);
                // the stage is free (here, and for the multicast, in every peer) once these products are done
                if (CL == 1)
                    mma_commit(&empty[s]);
                else
                    mma_commit_mc(&empty[s], (uint16_t)((1u << CL) - 1));
            }
            if (ok) mma_commit(&tfull[b]);
        }
        *consumed_s = it;
        __threadfence_block();
        // tensor memory is released only after every product issued has completed
        mma_commit(drain);
        if (!mbar_wait(drain, 0)) atomicOr(err, 8);
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31; waits and
        // decisions are taken by lane 0 so the warp stays converged for the
        // .sync.aligned loads
        const int q = warp & 3;
        float vmax = 0.f;
        int lt = 0;
        for (int t = cid; t < tiles; t += clusters, ++lt) {
            const int b = lt & 1;
            int go = 0;
            if (lane == 0) {
                const bool ok = mbar_wait(&tfull[b], (lt >> 1) & 1);
                if (!ok) atomicOr(err, 16);
                go = (ok && *failed_s == 0) ? 1 : 0;
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) break;
            fence_after();
            const int m0 = ((t % mgroups) * CL + rank) * BM, n0 = (t / mgroups) * BN;
            const int row = m0 + 32 * q + lane;
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld32(tbase + (uint32_t)(b * TMEM_COLS) + ((uint32_t)(32 * q) << 16) + 32 * c, v);
                if (row < rows) {
                    float *dst = C + (size_t)row * ldc + n0 + 32 * c;   // 32-byte aligned: ldc, n0 multiples of 256
#pragma unroll
                    for (int i = 0; i < 4; ++i) st_v8(dst + 8 * i, &v[8 * i]);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (n0 + 32 * c + 4 * i < vcols) vmax = fmaxf(vmax, v[4 * i] * v[4 * i] + v[4 * i + 1] * v[4 * i + 1]);
                }
            }
            // the loads above have completed (tcgen05.wait::ld); hand the buffer back
            fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[b])) : "memory");
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if (lane == 0 && vmax > 0.f) atomicMax(maxbits, __float_as_uint(vmax));
    }
    fence_before();
    __syncthreads();
    // on an error, wait (bounded, each) for loads issued but never consumed
    if (tid == 0 && *issued_s > *consumed_s) {
        for (int it = *consumed_s; it < *issued_s; ++it)
            if (!mbar_wait(&full[it % STAGES], (it / STAGES) & 1)) atomicOr(err, 32);
    }
    __syncthreads();
    // no CTA leaves while a peer may still deliver to its shared memory
    if (CL > 1) cluster_sync();
    fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(2 * TMEM_COLS) : "memory");
    }
}

// Pair form of the contraction: a cluster of two CTAs computes 256 x 256
// output tiles with one tcgen05.mma of M = 256 (cta_group::2) issued by the
// even CTA; each CTA loads its own 128 rows of A and its 128 rows of the basis
// tile (half of the N = 256 columns), so a stage is 32 KB per SM and six
// stages fit.  Loads of both CTAs complete on the even CTA's barrier; the
// products' completion is signalled to both CTAs (stage free, accumulator
// ready); each CTA reads back its own 128 rows from its tensor memory and
// tells the even CTA when the buffer is free.  Waits are bounded as in
// k_tc_gemm.
constexpr int P_STAGES = 6;
constexpr int P_STAGE = A_TILE + B_TILE / 2;   // 32 KB per CTA
constexpr size_t SMEM_PAIR = 1024 + (size_t)P_STAGES * P_STAGE + 256;

template <bool TF32>
__global__ void __launch_bounds__(THREADS, 1)
k_tc_gemm_pair(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
               const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1, float *__restrict__ C,
               int rows, int ldc, int vcols, int mtiles, int ntiles, int ktiles, int passes,
               unsigned *__restrict__ maxbits, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + P_STAGES * P_STAGE);
    uint64_t *empty = full + P_STAGES;
    uint64_t *tfull = empty + P_STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *issued_s = (volatile int *)(tmem_slot + 1);
    volatile int *consumed_s = issued_s + 1;
    volatile int *failed_s = issued_s + 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rank = (int)cluster_rank();
    const bool leader = rank == 0;
    const int cid = blockIdx.x >> 1, clusters = gridDim.x >> 1;
    const int mpairs = mtiles >> 1;
    const int tiles = mpairs * ntiles;
    const int per_tile = ktiles * passes;
    constexpr int KEL = TF32 ? 32 : 64;
    constexpr uint32_t ID = (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) |
                            ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);

    if (tid == 0) {
        for (int i = 0; i < P_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);   // four read-back warps in each CTA of the pair
        }
        mbar_init(drain, 1);
        *issued_s = 0;
        *consumed_s = 0;
        *failed_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(2 * TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    cluster_sync();
    fence_after();
    const uint32_t tbase = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer (both CTAs): own A rows and own half of the basis tile, counted on the even CTA's barrier
        int it = 0;
        bool ok = true;
        for (int t = cid; t < tiles && ok; t += clusters) {
            const int m0 = ((t % mpairs) * 2 + rank) * BM, n0 = (t / mpairs) * BN + rank * (BN / 2);
            for (int j = 0; j < per_tile; ++j, ++it) {
                const int s = it % P_STAGES;
                if (it >= P_STAGES && !mbar_wait_cluster(&empty[s], ((it / P_STAGES) & 1) ^ 1)) {
                    atomicOr(err, 1);
                    *failed_s = 1;
                    ok = false;
                    break;
                }
                const int pass = j / ktiles, kt = j % ktiles;
                const CUtensorMap *ma = (pass == 2) ? &tmA1 : &tmA0;
                const CUtensorMap *mb = (pass == 1) ? &tmB1 : &tmB0;
                uint8_t *sa = smem + s * P_STAGE, *sb = sa + A_TILE;
                if (leader) mbar_expect_tx(&full[s], 2 * P_STAGE);
                const uint32_t fb = mapa(su32(&full[s]), 0);
                tma_2d_pair(sa, ma, fb, kt * KEL, m0);
                tma_2d_pair(sb, mb, fb, kt * KEL, n0);
            }
        }
        *issued_s = it;
    } else if (warp == 1 && lane == 0 && leader) {
        // MMA issuer (even CTA)
        int it = 0, lt = 0;
        bool ok = true;
        for (int t = cid; t < tiles && ok; t += clusters, ++lt) {
            const int b = lt & 1;
            if (lt >= 2 && !mbar_wait_cluster(&tempty[b], ((lt >> 1) & 1) ^ 1)) {
                atomicOr(err, 2);
                *failed_s = 1;
                break;
            }
            fence_after();
            const uint32_t dt = tbase + (uint32_t)(b * TMEM_COLS);
            for (int j = 0; j < per_tile; ++j, ++it) {
                const int s = it % P_STAGES;
                if (!mbar_wait_cluster(&full[s], (it / P_STAGES) & 1)) {
                    atomicOr(err, 4);
                    *failed_s = 1;
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t sa = su32(smem + s * P_STAGE), sb = sa + A_TILE;
#pragma unroll
                for (int k = 0; k < KB / 32; ++k)
                    mma_pair<TF32>(dt, sdesc(sa + 32 * k), sdesc(sb + 32 * k), ID, (j > 0 || k > 0) ? 1u : 0u);
                mma_commit_pair(&empty[s]);
            }
            if (ok) mma_commit_pair(&tfull[b]);
        }
        *consumed_s = it;
        __threadfence_block();
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(drain))
                     : "memory");
        if (!mbar_wait(drain, 0)) atomicOr(err, 8);
    } else if (warp >= 2) {
        // read-back (both CTAs): this CTA's 128 rows of the pair's tile
        const int q = warp & 3;
        float vmax = 0.f;
        int lt = 0;
        const uint32_t te0 = mapa(su32(&tempty[0]), 0), te1 = mapa(su32(&tempty[1]), 0);
        for (int t = cid; t < tiles; t += clusters, ++lt) {
            const int b = lt & 1;
            int go = 0;
            if (lane == 0) {
                const bool okw = mbar_wait_cluster(&tfull[b], (lt >> 1) & 1);
                if (!okw) atomicOr(err, 16);
                go = (okw && *failed_s == 0) ? 1 : 0;
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) break;
            fence_after();
            const int m0 = ((t % mpairs) * 2 + rank) * BM, n0 = (t / mpairs) * BN;
            const int row = m0 + 32 * q + lane;
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld32(tbase + (uint32_t)(b * TMEM_COLS) + ((uint32_t)(32 * q) << 16) + 32 * c, v);
                if (row < rows) {
                    float *dst = C + (size_t)row * ldc + n0 + 32 * c;
#pragma unroll
                    for (int i = 0; i < 4; ++i) st_v8(dst + 8 * i, &v[8 * i]);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (n0 + 32 * c + 4 * i < vcols) vmax = fmaxf(vmax, v[4 * i] * v[4 * i] + v[4 * i + 1] * v[4 * i + 1]);
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(b ? te1 : te0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if (lane == 0 && vmax > 0.f) atomicMax(maxbits, __float_as_uint(vmax));
    }
    fence_before();
    __syncthreads();
    // on an error, wait (bounded) for this CTA's loads issued but never consumed
    // (the even CTA's barrier counts both CTAs' loads; only it can wait on them)
    if (tid == 0 && leader && *issued_s > *consumed_s) {
        for (int it = *consumed_s; it < *issued_s; ++it)
            if (!mbar_wait(&full[it % P_STAGES], (it / P_STAGES) & 1)) {
                atomicOr(err, 32);
                break;
            }
    }
    __syncthreads();
    cluster_sync();   // no CTA leaves while its peer may still write to it or read its tensor memory
    fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(2 * TMEM_COLS) : "memory");
    }
}

// zero-padded signal for the Hankel rows: xp[q] = x[q - M] (0 outside [0, n)),
// as BF16 hi and lo parts or as TF32 (rounded to nearest)
__global__ void k_tc_prep_x(const float *__restrict__ x, int64_t n, int M, int64_t len, int tf32,
                            __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo, float *__restrict__ f32,
                            unsigned *__restrict__ maxbits) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *maxbits = 0u;   // the contraction's running max |S^g|^2
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < len; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = q - M;
        const float v = (p >= 0 && p < n) ? x[p] : 0.f;
        if (tf32) {
            uint32_t r;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
            f32[q] = __uint_as_float(r);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[q] = h;
            lo[q] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// explicit Hankel copy A[m, j] = xp[m hop + j] (used when overlapping-row tensor maps are refused)
template <class T>
__global__ void k_tc_hankel(const T *__restrict__ xp, int hop, int64_t rows, int kpad, T *__restrict__ A) {
    const int64_t total = rows * (int64_t)kpad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / kpad, j = i % kpad;
        A[i] = xp[m * hop + j];
    }
}

// per frame: the FFT form's epilogue on the contraction's S^g, S^g' (MODE_T,
// MODE_STFT, MODE_MAP as in k_forward).  The CTA's frames m = blockIdx.x +
// i gridDim.x stream through two shared-memory row buffers filled by bulk
// copies, so the next frame's row arrives while this one is reassigned and
// written out.  With maxbits (relative thresholds) every CTA derives the
// call's scalars from the contraction's max |S^g|^2 itself; otherwise they
// come from sc.  Waits are bounded; on expiry the CTA records it in *err,
// drains its copies and stops.
template <int MODE>
__global__ void __launch_bounds__(256)
k_tc_band(SstDev d, const float *__restrict__ C, int ldc, const SstScalars *__restrict__ sc,
          const unsigned *__restrict__ maxbits, float frac2, float2 *__restrict__ out0, void *__restrict__ out1,
          int *__restrict__ err) {
    extern __shared__ uint4 smem_band[];
    const int stride = tacc_stride(d.nbo);
    const uint32_t rowbytes = 16u * (uint32_t)d.nb;
    const int tacc_words = MODE == MODE_T ? 4 * stride : 0;
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem_band);
    float4 *rows = reinterpret_cast<float4 *>(acc + tacc_words);          // 2 x nb float4
    uint64_t *bar = reinterpret_cast<uint64_t *>(rows + 2 * d.nb);         // 2 mbarriers
    volatile int *stop = reinterpret_cast<volatile int *>(bar + 2);
    const int tid = threadIdx.x;
    FwdScale fs;
    if (maxbits) {
        const SstScalars s = scalars_from_max(__uint_as_float(*maxbits), frac2, 0, 1.f, d.log2_nb);
        fs.gamma2 = s.gamma2;
        fs.s1 = s.s1; fs.s2 = s.s2; fs.r1 = s.r1; fs.r2 = s.r2;
    } else {
        fs = fwd_scale(d, sc, MODE == MODE_T);
    }
    const int64_t mine = (d.F - blockIdx.x + gridDim.x - 1) / gridDim.x;   // frames of this CTA
    for (int i = tid; i < tacc_words; i += blockDim.x) acc[i] = 0u;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int j = 0; j < 2 && j < mine; ++j) {
            mbar_expect_tx(&bar[j], rowbytes);
            bulk_g2s(rows + j * d.nb, C + (size_t)(blockIdx.x + (int64_t)j * gridDim.x) * ldc, rowbytes, &bar[j]);
        }
    int64_t i = 0;
    for (; i < mine; ++i) {
        const int b = (int)(i & 1);
        const int64_t m = blockIdx.x + i * gridDim.x;
        if (tid == 0 && !mbar_wait(&bar[b], (uint32_t)((i >> 1) & 1))) {
            atomicOr(err, 64);
            *stop = 1;
        }
        __syncthreads();
        if (*stop) break;
        const float4 *row = rows + b * d.nb;
        for (int kk = tid; kk < d.nb; kk += blockDim.x) {
            const float4 c = row[kk];
            const int k = d.k_lo + kk;
            const float2 V = make_float2(c.x, c.y), Vd = make_float2(c.z, c.w);
            const size_t o = (size_t)m * d.nb + kk;
            if (MODE == MODE_STFT) {
                out0[o] = V;
                reinterpret_cast<float2 *>(out1)[o] = make_float2(Vd.x * d.dscale, Vd.y * d.dscale);
                continue;
            }
            const float mag2 = V.x * V.x + V.y * V.y;
            // reassignment offset in bins: -(Nf / 2 pi) Im(S^g' / S^g)   (Eq. 13)
            const float delta = -d.c_if * ((Vd.y * V.x - Vd.x * V.y) / mag2);
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
                continue;
            }
            if (l >= 0) tacc_add(acc, stride, l, V, fs);
        }
        __syncthreads();   // row buffer b read, accumulators complete
        if (tid == 0 && i + 2 < mine) {
            mbar_expect_tx(&bar[b], rowbytes);
            bulk_g2s(rows + b * d.nb, C + (size_t)(m + 2 * (int64_t)gridDim.x) * ldc, rowbytes, &bar[b]);
        }
        if (MODE == MODE_T) {
            float2 *Trow = out0 + (size_t)trow_of(d, m) * d.nbo;
            for (int q = tid; 4 * q < d.nbo; q += blockDim.x) tacc_take4(acc, stride, q, d.nbo, Trow, fs);
            __syncthreads();
        }
    }
    // after an early stop: copies issued for frames i, i + 1 may still be in flight
    if (tid == 0 && i < mine) {
        for (int64_t j = i; j < mine && j < i + 2; ++j)
            if (!mbar_wait(&bar[j & 1], (uint32_t)((j >> 1) & 1))) atomicOr(err, 128);
    }
}

// dynamic shared memory of k_tc_band: accumulators, two row buffers, barriers
template <int MODE>
size_t tc_band_smem(const SstDev &d) {
    return (MODE == MODE_T ? tacc_bytes(d.nbo) : 0) + 32 * (size_t)d.nb + 32;
}

}  // namespace tc
}  // namespace sst

using namespace sst;
using namespace sst::tc;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct sst_tc_plan {
    sst_plan_t base = nullptr;
    int form = 0;
    bool hankel = false;
    int kpad = 0, ncols = 0, npad = 0;
    int64_t fpad = 0, xlen = 0;
    void *dmem = nullptr;
    void *xp0 = nullptr, *xp1 = nullptr;     // padded signal (hi, lo) or FP32
    void *A0 = nullptr, *A1 = nullptr;       // explicit Hankel copies when needed
    void *B0 = nullptr, *B1 = nullptr;       // basis (hi, lo) or FP32
    float *C = nullptr;                      // contraction output, fpad x npad
    int *err = nullptr;
    float *partial = nullptr;
    SstScalars *sc = nullptr;
    CUtensorMap tA0, tA1;
    CUtensorMap tB[3][2];                    // basis (hi, lo) with a box of BN / CL rows, CL = 1, 2, 4
    int cl = 1;                              // CTAs per cluster sharing the basis tile; 0: CTA pairs
    int grid[4] = {0, 0, 0, 0};              // persistent grid per variant (cluster 1, 2, 4, pair)
    bool withhold = false;                   // test hook, see sst_tc_plan_test_withhold
};

namespace {

typedef void (*GemmFn)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap, float *, int, int,
                       int, int, int, int, int, unsigned *, int *);

// cl: 1, 2, 4 (k_tc_gemm with that multicast cluster) or 0 (k_tc_gemm_pair)
GemmFn gemm_fn(bool tf32, int cl) {
    if (cl == 0) return tf32 ? k_tc_gemm_pair<true> : k_tc_gemm_pair<false>;
    if (tf32) return cl == 4 ? k_tc_gemm<true, 4> : cl == 2 ? k_tc_gemm<true, 2> : k_tc_gemm<true, 1>;
    return cl == 4 ? k_tc_gemm<false, 4> : cl == 2 ? k_tc_gemm<false, 2> : k_tc_gemm<false, 1>;
}
int variant_index(int cl) { return cl == 0 ? 3 : cl == 4 ? 2 : cl == 2 ? 1 : 0; }
int variant_cl(int vi) { return vi == 3 ? 0 : 1 << vi; }
int variant_ctas(int cl) { return cl == 0 ? 2 : cl; }    // CTAs per cluster

cudaLaunchConfig_t gemm_config(int grid, int cl, cudaStream_t st, cudaLaunchAttribute *at) {
    cudaLaunchConfig_t cfg = {};
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = variant_ctas(cl);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = cl == 0 ? SMEM_PAIR : SMEM;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

bool encode(CUtensorMap *m, bool tf32, void *base, uint64_t dim0, uint64_t dim1, uint64_t stride_bytes, uint32_t box1) {
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {dim0, dim1};
    const cuuint64_t strides[1] = {stride_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(tf32 ? 32 : 64), box1};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

uint16_t bf16_bits(float v) {
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    uint16_t r;
    memcpy(&r, &b, 2);
    return r;
}
// FP32 rounded to TF32 (10 fraction bits), to nearest with ties away from zero
float tf32_round(float v) {
    uint32_t u;
    memcpy(&u, &v, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    memcpy(&v, &u, 4);
    return v;
}
// a BF16 bit pattern's value: BF16 is the upper half of an FP32 (exact)
float bf16_val(uint16_t r) {
    const uint32_t u = (uint32_t)r << 16;
    float v;
    memcpy(&v, &u, 4);
    return v;
}

}  // namespace

SST_API sst_status sst_tc_plan_create(sst_plan_t base, int32_t form, sst_tc_plan_t *out) {
    SST_NVTX_RANGE();
    if (!out) return fail(SST_EINVAL, "out is NULL");
    *out = nullptr;
    if (!base) return fail(SST_EINVAL, "base plan is NULL");
    if (form != SST_FORM_BF16 && form != SST_FORM_BF16X3 && form != SST_FORM_TF32)
        return fail(SST_EINVAL, "unknown tensor form %d", form);
    if (!encoder()) return fail(SST_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    const SstDev &d = base->d;
    const bool tf32 = form == SST_FORM_TF32;
    const int esz = tf32 ? 4 : 2;
    const int kel = KB / esz;
    sst_tc_plan *t = new (std::nothrow) sst_tc_plan();
    if (!t) return fail(SST_ENOMEM, "host allocation failed");
    t->base = base;
    t->form = form;
    t->kpad = (d.L + kel - 1) / kel * kel;
    t->ncols = 4 * d.nb;
    t->npad = (t->ncols + BN - 1) / BN * BN;
    t->fpad = (d.F + 4 * BM - 1) / (4 * BM) * (4 * BM);   // whole clusters of up to 4 row blocks
    t->xlen = (t->fpad - 1) * d.hop + t->kpad;
    // FP64 basis: row 4 kk + c, column j (K-major); s g' as in the FFT form
    const int M = d.M, nf = d.nf;
    const std::vector<double> &g = base->g64, &dg = base->dgs64;
    const size_t belems = (size_t)t->npad * t->kpad;
    std::vector<uint16_t> bh, bl;
    std::vector<float> bf;
    if (tf32) bf.assign(belems, 0.f);
    else { bh.assign(belems, 0); bl.assign(belems, 0); }
    for (int kk = 0; kk < d.nb; ++kk) {
        const int64_t k = d.k_lo + kk;
        for (int j = 0; j < d.L; ++j) {
            const int64_t tt = (int64_t)j - M;
            const int64_t r = ((k * tt) % nf + nf) % nf;
            const double a = 2.0 * M_PI * (double)r / (double)nf;
            const double c = std::cos(a), s = std::sin(a);
            const double v[4] = {g[j] * c, -g[j] * s, dg[j] * c, -dg[j] * s};
            for (int q = 0; q < 4; ++q) {
                const size_t idx = (size_t)(4 * kk + q) * t->kpad + j;
                if (tf32) {
                    bf[idx] = tf32_round((float)v[q]);
                } else {
                    const uint16_t h = bf16_bits((float)v[q]);
                    bh[idx] = h;
                    bl[idx] = bf16_bits((float)(v[q] - (double)bf16_val(h)));
                }
            }
        }
    }
    // device buffers: xp0, xp1, B0, B1, A0, A1 (maybe), C, err, partial, scalars
    auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
    const size_t xbytes = al((size_t)t->xlen * esz), bbytes = al(belems * esz);
    const size_t abytes = al((size_t)t->fpad * t->kpad * esz), cbytes = al((size_t)t->fpad * t->npad * sizeof(float));
    const int two = tf32 ? 1 : 2;
    const size_t total = two * xbytes + two * bbytes + two * abytes + cbytes + 1024 + al(sizeof(float) * 4096) + 1024;
    if (cudaMalloc(&t->dmem, total) != cudaSuccess) {
        delete t;
        return fail(SST_ENOMEM, "tensor-form buffers of %zu bytes", total);
    }
    char *p = (char *)t->dmem;
    t->xp0 = p; p += xbytes;
    if (!tf32) { t->xp1 = p; p += xbytes; }
    t->B0 = p; p += bbytes;
    if (!tf32) { t->B1 = p; p += bbytes; }
    t->A0 = p; p += abytes;
    if (!tf32) { t->A1 = p; p += abytes; }
    t->C = (float *)p; p += cbytes;
    t->err = (int *)p; p += 1024;
    t->partial = (float *)p; p += al(sizeof(float) * 4096);
    t->sc = (SstScalars *)p;
    cudaError_t e = tf32 ? cudaMemcpy(t->B0, bf.data(), belems * 4, cudaMemcpyHostToDevice)
                         : cudaMemcpy(t->B0, bh.data(), belems * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tf32) e = cudaMemcpy(t->B1, bl.data(), belems * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(t->err, 0, 1024);   // error word, test-hook word
    if (e != cudaSuccess) {
        cudaFree(t->dmem);
        delete t;
        return cuda_fail(e, "tensor-form upload");
    }
    // tensor maps: B is [npad rows x kpad]; A is the Hankel view of xp (rows hop apart), else explicit copies
    bool ok = true;
    for (int ci = 0; ci < 3; ++ci) {
        ok = ok && encode(&t->tB[ci][0], tf32, t->B0, t->kpad, t->npad, (uint64_t)t->kpad * esz, BN >> ci);
        ok = ok && encode(&t->tB[ci][1], tf32, tf32 ? t->B0 : t->B1, t->kpad, t->npad, (uint64_t)t->kpad * esz,
                          BN >> ci);
    }
    if (!ok) {
        cudaFree(t->dmem);
        delete t;
        return fail(SST_EUNSUPPORTED, "tensor map of the basis refused");
    }
    const uint64_t hstride = (uint64_t)d.hop * esz;
    t->hankel = (hstride % 16 == 0) && encode(&t->tA0, tf32, t->xp0, t->kpad, t->fpad, hstride, BM) &&
                encode(&t->tA1, tf32, tf32 ? t->xp0 : t->xp1, t->kpad, t->fpad, hstride, BM);
    if (!t->hankel) {
        ok = encode(&t->tA0, tf32, t->A0, t->kpad, t->fpad, (uint64_t)t->kpad * esz, BM) &&
             encode(&t->tA1, tf32, tf32 ? t->A0 : t->A1, t->kpad, t->fpad, (uint64_t)t->kpad * esz, BM);
        if (!ok) {
            cudaFree(t->dmem);
            delete t;
            return fail(SST_EUNSUPPORTED, "tensor map of the frames refused");
        }
    }
    e = cudaSuccess;
    for (int vi = 0; vi < 4 && e == cudaSuccess; ++vi) {
        const int cl = variant_cl(vi);
        e = cudaFuncSetAttribute(gemm_fn(tf32, cl), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(cl == 0 ? SMEM_PAIR : SMEM));
    }
    // persistent grids: one CTA per SM, whole clusters only, no more clusters than tiles
    const int mtiles = (int)(t->fpad / BM), ntiles = t->npad / BN;
    for (int vi = 0; vi < 4 && e == cudaSuccess; ++vi) {
        const int cl = variant_cl(vi), ctas = variant_ctas(cl);
        int clusters = base->num_sms / ctas;
        if (ctas > 1) {
            cudaLaunchAttribute at[1];
            cudaLaunchConfig_t cfg = gemm_config(ctas * clusters, cl, nullptr, at);
            int active = 0;
            e = cudaOccupancyMaxActiveClusters(&active, gemm_fn(tf32, cl), &cfg);
            if (e != cudaSuccess) break;
            clusters = std::min(clusters, active);
        }
        clusters = std::min(clusters, (mtiles / ctas) * ntiles);
        t->grid[vi] = std::max(clusters, 0) * ctas;
    }
    t->cl = 1;
    // the epilogue's accumulators and row buffers; the limit is only ever
    // raised, so plans with different band widths can share the kernels
    {
        static std::mutex mu;
        static size_t band_max[3] = {48 * 1024, 48 * 1024, 48 * 1024};
        const size_t need[3] = {tc_band_smem<MODE_T>(d), tc_band_smem<MODE_STFT>(d), tc_band_smem<MODE_MAP>(d)};
        const void *fns[3] = {(const void *)k_tc_band<MODE_T>, (const void *)k_tc_band<MODE_STFT>,
                              (const void *)k_tc_band<MODE_MAP>};
        std::lock_guard<std::mutex> lk(mu);
        for (int i = 0; i < 3 && e == cudaSuccess; ++i)
            if (need[i] > band_max[i]) {
                e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need[i]);
                if (e == cudaSuccess) band_max[i] = need[i];
            }
    }
    if (e != cudaSuccess) {
        cudaFree(t->dmem);
        delete t;
        return cuda_fail(e, "tensor-form kernel attributes");
    }
    *out = t;
    return SST_OK;
}

SST_API void sst_tc_plan_destroy(sst_tc_plan_t t) {
    if (!t) return;
    if (t->dmem) cudaFree(t->dmem);
    delete t;
}

SST_API sst_status sst_tc_plan_query(sst_tc_plan_t t, int32_t *hankel_view, int64_t *gemm_flops, int32_t *cluster) {
    if (!t) return fail(SST_EINVAL, "plan is NULL");
    if (cluster) *cluster = t->cl;
    if (hankel_view) *hankel_view = t->hankel ? 1 : 0;
    if (gemm_flops)
        *gemm_flops = 2LL * t->base->d.F * (int64_t)t->ncols * t->base->d.L * (t->form == SST_FORM_BF16X3 ? 3 : 1);
    return SST_OK;
}

SST_API sst_status sst_tc_check(sst_tc_plan_t t, void *stream);

// the contraction: signal prep (and explicit Hankel copy when needed), GEMM, error check
static sst_status tc_contract(sst_tc_plan_t t, const float *x, cudaStream_t st) {
    const SstDev &d = t->base->d;
    const bool tf32 = t->form == SST_FORM_TF32;
    const int blocks = (int)std::min<int64_t>((t->xlen + 255) / 256, 4096);
    SST_LAUNCHED_K(PK_OTHER, st,
                   (k_tc_prep_x<<<blocks, 256, 0, st>>>(x, d.n, d.M, t->xlen, tf32 ? 1 : 0,
                                                        tf32 ? nullptr : (__nv_bfloat16 *)t->xp0,
                                                        tf32 ? nullptr : (__nv_bfloat16 *)t->xp1,
                                                        tf32 ? (float *)t->xp0 : nullptr, (unsigned *)t->partial),
                    cudaGetLastError()),
                   "tensor-form signal prep");
    if (!t->hankel) {
        const int hb = (int)std::min<int64_t>((t->fpad * t->kpad + 255) / 256, 8192);
        if (tf32) {
            SST_LAUNCHED_K(PK_OTHER, st,
                           (k_tc_hankel<float><<<hb, 256, 0, st>>>((const float *)t->xp0, d.hop, t->fpad, t->kpad, (float *)t->A0),
                            cudaGetLastError()),
                           "hankel copy");
        } else {
            SST_LAUNCHED_K(PK_OTHER, st,
                           (k_tc_hankel<__nv_bfloat16><<<hb, 256, 0, st>>>((const __nv_bfloat16 *)t->xp0, d.hop, t->fpad,
                                                                           t->kpad, (__nv_bfloat16 *)t->A0),
                            cudaGetLastError()),
                           "hankel copy");
            SST_LAUNCHED_K(PK_OTHER, st,
                           (k_tc_hankel<__nv_bfloat16><<<hb, 256, 0, st>>>((const __nv_bfloat16 *)t->xp1, d.hop, t->fpad,
                                                                           t->kpad, (__nv_bfloat16 *)t->A1),
                            cudaGetLastError()),
                           "hankel copy");
        }
    }
    const int ktiles = t->kpad / (KB / (tf32 ? 4 : 2));
    const int passes = t->form == SST_FORM_BF16X3 ? 3 : 1;
    const int mtiles = (int)(t->fpad / BM), ntiles = t->npad / BN;
    const int vi = variant_index(t->cl);
    const int bi = t->cl == 0 ? 1 : (t->cl == 4 ? 2 : t->cl == 2 ? 1 : 0);   // basis box: BN / (CTAs sharing it)
    if (t->withhold) SST_CU(cudaMemsetAsync(t->err + 1, 0xff, sizeof(int), st), "test hook");
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = gemm_config(t->grid[vi], t->cl, st, at);
    SST_LAUNCHED_K(PK_STFT, st,
                   cudaLaunchKernelEx(&cfg, gemm_fn(tf32, t->cl), t->tA0, t->tA1, t->tB[bi][0], t->tB[bi][1], t->C,
                                      (int)d.F, t->npad, t->ncols, mtiles, ntiles, ktiles, passes,
                                      (unsigned *)t->partial, t->err),
                   "tensor contraction");
    if (t->withhold) {
        SST_CU(cudaMemsetAsync(t->err + 1, 0, sizeof(int), st), "test hook");
        t->withhold = false;
    }
    return SST_OK;
}

SST_API sst_status sst_tc_plan_test_withhold(sst_tc_plan_t t) {
    if (!t) return fail(SST_EINVAL, "plan is NULL");
    if (t->cl != 1) return fail(SST_EINVAL, "the test hook needs cluster 1");
    t->withhold = true;
    return SST_OK;
}

SST_API sst_status sst_tc_plan_tune(sst_tc_plan_t t, const float *x_dev, int64_t n, void *stream, int32_t *cluster,
                                    float *ms_out) {
    SST_NVTX_RANGE();
    if (!t) return fail(SST_EINVAL, "plan is NULL");
    if (!x_dev) return fail(SST_EINVAL, "input pointer is NULL");
    if (n != t->base->d.n) return fail(SST_EINVAL, "n = %lld differs from the plan's n", (long long)n);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    SST_CU(cudaEventCreate(&a), "event");
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(SST_ECUDA, "event");
    }
    const int keep = t->cl;
    int best = -1;
    float best_ms = 0.f;
    sst_status s = SST_OK;
    for (int vi = 0; vi < 4 && s == SST_OK; ++vi) {
        if (t->grid[vi] <= 0) continue;
        t->cl = variant_cl(vi);
        float ms = 0.f;
        // one untimed run, then the best of three
        for (int r = 0; r < 4 && s == SST_OK; ++r) {
            if (cudaEventRecord(a, st) != cudaSuccess) { s = fail(SST_ECUDA, "event record"); break; }
            s = tc_contract(t, x_dev, st);
            if (s != SST_OK) break;
            if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
                s = fail(SST_ECUDA, "event timing");
                break;
            }
            float e = 0.f;
            cudaEventElapsedTime(&e, a, b);
            if (r == 1 || (r > 1 && e < ms)) ms = e;
        }
        if (s == SST_OK && (best < 0 || ms < best_ms)) {
            best = t->cl;
            best_ms = ms;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != SST_OK) {
        t->cl = keep;
        return s;
    }
    if ((s = sst_tc_check(t, stream)) != SST_OK) {
        t->cl = keep;
        return s;
    }
    t->cl = best >= 0 ? best : keep;
    if (cluster) *cluster = t->cl;
    if (ms_out) *ms_out = best_ms;
    return SST_OK;
}

SST_API sst_status sst_tc_plan_set_cluster(sst_tc_plan_t t, int32_t cluster) {
    if (!t) return fail(SST_EINVAL, "plan is NULL");
    if (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4)
        return fail(SST_EINVAL, "cluster must be 1, 2, 4 (multicast) or 0 (CTA pairs)");
    if (t->grid[variant_index(cluster)] <= 0)
        return fail(SST_EUNSUPPORTED, "no cluster of this kind (%d) fits this device", cluster);
    t->cl = cluster;
    return SST_OK;
}

SST_API sst_status sst_tc_check(sst_tc_plan_t t, void *stream) {
    SST_NVTX_RANGE();
    if (!t) return fail(SST_EINVAL, "plan is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    SST_CU(cudaMemcpyAsync(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost, st), "error word");
    SST_CU(cudaStreamSynchronize(st), "error word");
    if (h) {
        SST_CU(cudaMemsetAsync(t->err, 0, sizeof(int), st), "error word reset");
        SST_CU(cudaStreamSynchronize(st), "error word reset");
        return fail(SST_ETIMEOUT, "tensor contraction gave up waiting (site mask 0x%x)", h);
    }
    return SST_OK;
}

static sst_status tc_scalars(sst_tc_plan_t t, const float *x, cudaStream_t st) {
    const SstDev &d = t->base->d;
    if (d.relative) {
        // nothing to launch: the contraction's epilogue folded max |S^g|^2
        // into one word and every epilogue CTA derives gamma and the scale
    } else {
        const int grid = (int)std::min<int64_t>((d.n + 255) / 256, 1024);
        SST_LAUNCHED_K(PK_ABSMAX, st, launch_absx(x, d.n, t->partial + 1, grid, st), "absx launch");
        SST_LAUNCHED_K(PK_GAMMA, st,
                       launch_gamma(t->partial + 1, grid, t->base->gamma_frac2, 1, t->base->sum_abs_g, d.log2_nb,
                                    t->sc, nullptr, nullptr, st),
                       "gamma launch");
    }
    return SST_OK;
}

template <int MODE>
static sst_status tc_band(sst_tc_plan_t t, void *o0, void *o1, cudaStream_t st) {
    const SstDev &d = t->base->d;
    const size_t smem = tc_band_smem<MODE>(d);
    const int per_sm = std::max(1, std::min(8, (int)(200 * 1024 / smem)));
    const int grid = (int)std::min<int64_t>(d.F, (int64_t)t->base->num_sms * per_sm);
    const bool rel = d.relative && MODE != MODE_STFT;
    SST_LAUNCHED_K(MODE == MODE_T ? PK_FORWARD : (MODE == MODE_STFT ? PK_STFT : PK_MAP), st,
                   (k_tc_band<MODE><<<grid, 256, smem, st>>>(d, t->C, t->npad, t->sc,
                                                           rel ? (const unsigned *)t->partial : nullptr,
                                                           t->base->gamma_frac2, (float2 *)o0, o1, t->err),
                    cudaGetLastError()),
                   "tensor-form epilogue");
    return SST_OK;
}

static sst_status tc_check(sst_tc_plan_t t, const void *x, int64_t n) {
    if (!t) return fail(SST_EINVAL, "plan is NULL");
    if (!x) return fail(SST_EINVAL, "input pointer is NULL");
    if (n != t->base->d.n) return fail(SST_EINVAL, "n = %lld differs from the plan's n", (long long)n);
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != t->base->device) return fail(SST_EINVAL, "plan was created on device %d, current is %d", t->base->device, dev);
    return SST_OK;
}

SST_API sst_status sst_tc_forward(sst_tc_plan_t t, const float *x_dev, int64_t n, float *tfr_dev, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = tc_check(t, x_dev, n);
    if (s != SST_OK) return s;
    if (!tfr_dev) return fail(SST_EINVAL, "tfr pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = tc_contract(t, x_dev, st)) != SST_OK) return s;
    if ((s = tc_scalars(t, x_dev, st)) != SST_OK) return s;
    if ((s = tc_band<MODE_T>(t, tfr_dev, nullptr, st)) != SST_OK) return s;
    return SST_OK;
}

SST_API sst_status sst_tc_stft(sst_tc_plan_t t, const float *x_dev, int64_t n, float *V_dev, float *Vd_dev,
                               void *stream) {
    SST_NVTX_RANGE();
    sst_status s = tc_check(t, x_dev, n);
    if (s != SST_OK) return s;
    if (!V_dev || !Vd_dev) return fail(SST_EINVAL, "output pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = tc_contract(t, x_dev, st)) != SST_OK) return s;
    if ((s = tc_band<MODE_STFT>(t, V_dev, Vd_dev, st)) != SST_OK) return s;
    return SST_OK;
}

SST_API sst_status sst_tc_reassign_map(sst_tc_plan_t t, const float *x_dev, int64_t n, float *omega_dev,
                                       int32_t *dest_dev, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = tc_check(t, x_dev, n);
    if (s != SST_OK) return s;
    if (!omega_dev || !dest_dev) return fail(SST_EINVAL, "output pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = tc_contract(t, x_dev, st)) != SST_OK) return s;
    if ((s = tc_scalars(t, x_dev, st)) != SST_OK) return s;
    if ((s = tc_band<MODE_MAP>(t, omega_dev, dest_dev, st)) != SST_OK) return s;
    return SST_OK;
}

// the contraction alone (for timing): enqueue only, no synchronisation
SST_API sst_status sst_tc_contract(sst_tc_plan_t t, const float *x_dev, int64_t n, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = tc_check(t, x_dev, n);
    if (s != SST_OK) return s;
    return tc_contract(t, x_dev, (cudaStream_t)stream);
}
