/*
 * k_conv_tc.cu -- the separable far-part convolutions (Sec. V, Eqs. 31-32) on
 * the 5th-generation tensor cores: tcgen05.mma with operands staged in shared
 * memory by TMA and FP32 accumulators in tensor memory.
 *
 * Each 1D pass contracts the contiguous axis of its input against n x n
 * circulant matrices of the deconvolved Gaussians, one per term, and writes
 * its output with the axes rotated so that the next pass again contracts a
 * contiguous axis (every operand K-major):
 *
 *   pass x  A = rho  [lines (z, y)][x]                 B_j = K~x_j  (+ DC row)
 *           -> X[j][x][z][y]
 *   pass y  A = X_j  [lines (x, z)][y]                 B_j = K~y_j  (+ DC row)
 *           -> Y[y][x][j][z]
 *   pass z  A = Y    [lines (y, x)][(j, z)]            B   = [s_j K~z_j]_j (+ DC row)
 *           -> psi[z][y][x]            (the sum over terms is part of K)
 *
 * A 1D kernel is its zero-mean circulant part K~ plus its mean mu (Gaussians
 * wide compared with the box are almost constant, and the split keeps their
 * varying part accurate).  The mean acts through the row sum of A, which the
 * tensor core computes as one extra column: the "DC row" of B holds ones (x,
 * y passes) or the weights s_j mu_j (z pass); the epilogue adds mu_j times it.
 *
 * Precision: operands are split into high and low parts, A = A_hi + A_lo,
 * B = B_hi + B_lo, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in
 * FP32 (three MMAs per k-step): TF32x3 (10 + 10 mantissa bits per operand)
 * or BF16x3 (7 + 8).  Each epilogue writes the hi and lo parts of its output
 * for the next pass; the last writes FP32.
 *
 * CTA: 128 threads, one 128-line M tile, one N tile of NT <= 256 columns
 * (NT - 1 output columns and the DC column at most), the K loop in stages of
 * 128 bytes per row (32 TF32 or 64 BF16 values) through an S-stage TMA ring.
 * Warp 0 lane 0 issues the TMA loads, warp 1 owns the tensor memory and lane 0
 * of it issues the MMAs; all four warps run the epilogue (warp w reads TMEM
 * lanes 32w..32w+31, one line per thread).  Every wait is bounded in time:
 * on expiry the CTA raises the timeout bit of the status word, waits (again
 * bounded) for its copies in flight, frees its tensor memory and returns.
 * For tests, inject_wait_ns != 0 makes the MMA issuer first wait on a barrier
 * that no thread ever arrives at, bounded by that limit, so that this path
 * runs without any fault.
 */
#include <cuda.h>
#include <cuda_bf16.h>

#include "usr_internal.h"

namespace usr {

namespace {

constexpr int kTcThreads = 128;
constexpr int kRowBytes = 128;                      // one swizzle-128B row per stage
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

/*
 * Bounded wait for the phase of `parity`: false after limit_ns, or (when
 * abort_flag is given) as soon as another role of the CTA has aborted.
 */
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                          unsigned long long limit_ns = kWaitNs)
{
    const unsigned long long t0 = globaltimer();
    while (!mbar_try(bar, parity)) {
        if (abort_flag && *abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

/* Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart. */
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);           // start address
    d |= (uint64_t)1 << 16;                            // leading-dimension offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride-dimension offset: next 8-row group
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (BF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    #pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_round(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

/* Store the hi/lo split of v at index i of the pass output. */
template <bool BF16>
__device__ __forceinline__ void store_split(void* hi, void* lo, size_t i, float v)
{
    if (BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        static_cast<__nv_bfloat16*>(hi)[i] = h;
        static_cast<__nv_bfloat16*>(lo)[i] = l;
    } else {
        const float h = tf32_round(v);
        static_cast<float*>(hi)[i] = h;
        static_cast<float*>(lo)[i] = v - h;
    }
}

}  // namespace

template <bool BF16>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const __grid_constant__ CUtensorMap mA_hi,
                                                           const __grid_constant__ CUtensorMap mA_lo,
                                                           const __grid_constant__ CUtensorMap mB_hi,
                                                           const __grid_constant__ CUtensorMap mB_lo, ConvTcArgs g)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    constexpr int KMMA = BF16 ? 16 : 8;                // K of one MMA
    constexpr int KSTAGE = BF16 ? 64 : 32;             // K per 128-byte row
    constexpr int KSUB = KSTAGE / KMMA;                // MMAs per stage and operand pair (4)
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2 * kConvTcMaxStages + 2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128;
    const int batch = blockIdx.y, tile = blockIdx.z;
    const int S = g.stages, NT = g.NT;
    const uint32_t a_bytes = 128 * kRowBytes;
    const uint32_t b_bytes = (uint32_t)NT * kRowBytes;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    // 1024-byte aligned stage ring
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kConvTcMaxStages]);
    const uint32_t done = smem_u32(&bars[2 * kConvTcMaxStages]);
    const uint32_t never = smem_u32(&bars[2 * kConvTcMaxStages + 1]);   // no thread ever arrives here
    const int nk = (g.K + KSTAGE - 1) / KSTAGE;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"((uint32_t)g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    const int a_row = batch * g.a_rows_per_batch + m0;
    const int b_row = (batch * g.ntiles + tile) * NT;
    int issued = 0;
    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % S, use = kb / S;
            if (use > 0 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1, &abort_flag)) {
                atomicOr(g.status, 4);
                abort_flag = 1;
                break;
            }
            const uint32_t st = base + s * stage_bytes;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, stage_bytes);
            const int kc = kb * KSTAGE;
            tma_load_2d(st, &mA_hi, kc, a_row, fb);
            tma_load_2d(st + a_bytes, &mA_lo, kc, a_row, fb);
            tma_load_2d(st + 2 * a_bytes, &mB_hi, kc, b_row, fb);
            tma_load_2d(st + 2 * a_bytes + b_bytes, &mB_lo, kc, b_row, fb);
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        uint32_t idesc = (1u << 4)                                    // D: FP32
                         | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10)   // A, B: BF16 or TF32
                         | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        bool ok = true;
        if (g.inject_wait_ns && !mbar_wait(never, 0, &abort_flag, g.inject_wait_ns)) {
            // the test form of a wait that runs out: same abort path as a real one
            atomicOr(g.status, 4);
            abort_flag = 1;
            ok = false;
        }
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % S, use = kb / S;
            if (!mbar_wait(full0 + 8 * s, use & 1, &abort_flag)) {
                atomicOr(g.status, 4);
                abort_flag = 1;
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + s * stage_bytes;
            const uint64_t ah = sdesc(st), al = sdesc(st + a_bytes);
            const uint64_t bh = sdesc(st + 2 * a_bytes), bl = sdesc(st + 2 * a_bytes + b_bytes);
            #pragma unroll
            for (int k = 0; k < KSUB; ++k) {
                const uint64_t off = (uint64_t)((k * KMMA * (BF16 ? 2 : 4)) >> 4);   // bytes along the row
                const uint32_t first = (kb == 0 && k == 0) ? 0u : 1u;
                mma<BF16>(tmem, ah + off, bh + off, idesc, first);
                mma<BF16>(tmem, ah + off, bl + off, idesc, 1u);
                mma<BF16>(tmem, al + off, bh + off, idesc, 1u);
            }
            mma_commit(empty0 + 8 * s);            // the stage is free once these MMAs have read it
        }
        mma_commit(done);                          // accumulator complete (or in-flight MMAs drained)
    }
    __syncwarp();

    // epilogue: all four warps (the MMA issuer always commits `done`, so this
    // wait also drains MMAs still in flight after an abort)
    const bool have = mbar_wait(done, 0, nullptr);
    if (!have && threadIdx.x == 0) {
        atomicOr(g.status, 4);
        abort_flag = 1;
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have && !abort_flag) {
        const int r = warp * 32 + lane;
        const int line = m0 + r;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float v[16];
        // the DC column sits right after the tile's real columns
        const int dcc = g.cols;
        tmem_ld16(trow + (uint32_t)(dcc & ~15), v);
        float dc = 0.f;
        #pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i == (dcc & 15)) dc = v[i];
        const bool valid = line < g.lines;
        const int c_lo = tile * g.cols;
        float muj = 0.f;
        if (g.pass != 3) muj = g.mu[batch];
        int lx = 0, lz = 0;
        if (g.pass == 2) {
            lx = line / g.nz;
            lz = line - lx * g.nz;
        }
        for (int c0 = 0; c0 < g.cols; c0 += 16) {
            tmem_ld16(trow + (uint32_t)c0, v);
            if (!valid) continue;
            #pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = c0 + i;
                const int m = c_lo + c;
                if (c >= g.cols || m >= g.n_out) continue;
                if (g.pass == 1) {
                    const float val = fmaf(muj, dc, v[i]);
                    const size_t idx = (size_t)(batch * g.nx + m) * g.lines + line;
                    if (USR_IN_BOUNDS(idx, g.out_elems, g.status)) store_split<BF16>(g.out_hi, g.out_lo, idx, val);
                } else if (g.pass == 2) {
                    const float val = fmaf(muj, dc, v[i]);
                    const size_t idx = ((size_t)(m * g.nx + lx) * g.nterms + batch) * g.nz + lz;
                    if (USR_IN_BOUNDS(idx, g.out_elems, g.status)) store_split<BF16>(g.out_hi, g.out_lo, idx, val);
                } else {
                    const size_t idx = (size_t)m * g.lines + line;
                    if (USR_IN_BOUNDS(idx, g.out_elems, g.status)) static_cast<float*>(g.out_hi)[idx] = v[i] + dc;
                }
            }
        }
    }
    // teardown: make sure no copy is still landing in shared memory, then free TMEM
    if (warp == 0 && lane == 0 && abort_flag) {
        for (int kb = max(0, issued - S); kb < issued; ++kb) mbar_wait(full0 + 8 * (kb % S), (kb / S) & 1, nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)g.tmem_cols));
}

/* ------------------------------------------------------------------ host */

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    // looked up once, thread-safely (several serving threads configure contexts at once)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return nullptr;
    }();
    return fn;
}

}  // namespace

/* 2D tensor map over a row-major [rows][K] matrix, box [box_rows][128 bytes], 128-byte swizzle. */
usr_status make_tmap(CUtensorMap* m, const void* ptr, bool bf16, long long rows, int K, int box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return USR_ERR_CUDA;
    const int esz = bf16 ? 2 : 4;
    if (((uintptr_t)ptr & 15u) || ((long long)K * esz) % 16 != 0) return USR_ERR_BOX;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * esz};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? USR_OK : USR_ERR_CUDA;
}

size_t conv_tc_smem(const ConvTcArgs& g)
{
    return (size_t)g.stages * (2 * 128 + 2 * g.NT) * kRowBytes + 1024;
}

usr_status conv_tc_setup(bool bf16, size_t smem)
{
    cudaError_t e = bf16 ? cudaFuncSetAttribute(k_conv_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                         : cudaFuncSetAttribute(k_conv_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e == cudaSuccess ? USR_OK : USR_ERR_CUDA;
}

void launch_conv_tc(bool bf16, const ConvTcMaps& m, const ConvTcArgs& g, int batches, cudaStream_t st)
{
    dim3 grid((g.lines + 127) / 128, batches, g.ntiles);
    const size_t smem = (size_t)g.smem;
    if (bf16)
        launch_pdl(k_conv_tc<true>, grid, kTcThreads, smem, st, m.a_hi, m.a_lo, m.b_hi, m.b_lo, g);
    else
        launch_pdl(k_conv_tc<false>, grid, kTcThreads, smem, st, m.a_hi, m.a_lo, m.b_hi, m.b_lo, g);
}

}  // namespace usr
