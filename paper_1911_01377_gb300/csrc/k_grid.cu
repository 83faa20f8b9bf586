/*
 * k_grid.cu -- the particle-grid legs of the far part (Sec. V with Gaussian
 * spreading, the GSE scheme named in Sec. IV.A), atomic-free and
 * deterministic.  Both grid kernels work on blocks of cells: one CTA owns
 * kb_x x kb_y x kb_z cells of the sorted cell list and a shared-memory tile of
 * grid points covering the P^3 stencils of all their atoms.
 *
 *   spread   rho_g = sum_i q_i exp(-|g - r_i|^2 / (2 sigma_s^2)) (normalisation
 *            folded into the convolution scale).  The CTA's warps own disjoint
 *            sets of tile rows (y = warp mod 8) and every warp walks the
 *            block's atoms in sorted order, adding the stencil columns of its
 *            rows (one lane per column and group of planes) with plain
 *            shared-memory read-modify-writes: no atomics, and every tile point
 *            receives its terms in a fixed order.  The
 *            tile is stored whole to a tile buffer, and the block's tile sum
 *            is kept; the last CTA forms the grid mean (the k = 0 mode,
 *            dropped per Eq. 4) from those sums in block order.
 *   reduce   one thread per grid point adds the tiles that hold it, in block
 *            order, and subtracts the grid mean.
 *   gather   phi_far,i = sum_g w(g - r_i) psi_g and F_far,i = -q_i grad phi_far,i
 *            (the second spreading Gaussian of Eq. 32's 1/|S(k)|^2), per sorted
 *            atom, reading psi from global memory; contracts the stencil
 *            separably (z first, per (x, y) column); also psi's grid mean.
 *   combine  after the pair kernel: near + far + the self term -F(0) q_i in
 *            caller order, and E = 1/2 sum q_i phi_i and its parts
 *            (compensated FP32 within a warp, FP64 across warps and blocks).
 */
#include <cuda_bf16.h>

#include "usr_internal.h"

namespace usr {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 128;         // atoms whose weights are staged at once (spread)
constexpr int kGChunk = 128;        // atoms staged at once (gather)
constexpr int kMaxRows = 64;        // (cz, cy) rows of cells per block

__device__ __forceinline__ double warp_sum_d(double v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

/*
 * Compensated FP32 accumulation (Neumaier): s + c carries the sum to about FP32 rounding of the total,
 * independent of the number of terms.  FP64 is kept for the sums across threads: GB300's FP64 rate is
 * about 1/64 of FP32, so per-element FP64 arithmetic in these kernels cost more than their FP32 work.
 */
struct CSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s));
        s = t;
    }
    // a * b exactly, as the rounded product and its rounding error (fmaf gives the error exactly)
    __device__ __forceinline__ void add_product(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        add(p);
        add(fmaf(a, b, -p));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

/* A compensated sum over the warp (xor butterfly, FP32 with the error terms carried), as FP64: one conversion
   per warp instead of five FP64 additions per thread (GB300's FP64 pipe is narrow). Callers use lane 0's value. */
__device__ __forceinline__ double warp_sum_c(CSum cs)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s = __shfl_xor_sync(0xffffffffu, cs.s, o), c = __shfl_xor_sync(0xffffffffu, cs.c, o);
        cs.add(s);
        cs.c = __fadd_rn(cs.c, c);
    }
    return cs.value();
}

__device__ __forceinline__ float warp_sum_f(float v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

/* Periodic wrap of a grid index that lies within two periods of [0, n). */
__device__ __forceinline__ int wrap_once(int v, int n)
{
    if (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

/* Block coordinates, cell range and tile origin of CTA `bid`. */
struct BlockGeom {
    int c0[3], c1[3];
    int o[3];
};

__device__ __forceinline__ BlockGeom block_geom(const GridArgs& g, int bid)
{
    BlockGeom b;
    const int nb0 = g.tg.nbk[0], nb1 = g.tg.nbk[1];
    const int bc[3] = {bid % nb0, (bid / nb0) % nb1, bid / (nb0 * nb1)};
    #pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.c0[a] = bc[a] * g.tg.kb[a];
        b.c1[a] = min(g.box.nc[a], b.c0[a] + g.tg.kb[a]);
        b.o[a] = g.tab.org[a][bc[a]];
    }
    return b;
}

/*
 * The block's atoms are the x-runs of its (cz, cy) cell rows, contiguous in
 * the sorted array.  Fills rs/pre (row start, prefix count) and returns the
 * total.  Called by all threads; thread 0 writes, then a barrier.
 */
__device__ int block_rows(const GridArgs& g, const BlockGeom& bg, const int* __restrict__ cell_start, int* rs,
                          int* pre)
{
    const int ncx = g.box.nc[0], ncy = g.box.nc[1];
    const int ny = bg.c1[1] - bg.c0[1];
    const int nrows = ny * (bg.c1[2] - bg.c0[2]);
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int r = 0; r < nrows; ++r) {
            const int cz = bg.c0[2] + r / ny, cy = bg.c0[1] + r % ny;
            const int row = (cz * ncy + cy) * ncx;
            const int s = cell_start[row + bg.c0[0]], e = cell_start[row + bg.c1[0]];
            rs[r] = s;
            pre[r] = acc;
            acc += e - s;
        }
        pre[nrows] = acc;
    }
    __syncthreads();
    return pre[nrows];
}

/* Sorted-array index of the block's j-th atom. */
__device__ __forceinline__ int block_atom(int j, const int* rs, const int* pre)
{
    int r = 0;
    while (pre[r + 1] <= j) ++r;
    return rs[r] + (j - pre[r]);
}

}  // namespace

/* ------------------------------------------------------------------ spread */

template <int P>
__global__ void __launch_bounds__(kThreads, 2) k_spread(const float4* __restrict__ pos,
                                                        const int* __restrict__ cell_start, GridArgs g,
                                                        float* __restrict__ tilebuf, double* __restrict__ partial,
                                                        unsigned int* __restrict__ counter,
                                                        double* __restrict__ mean, int* __restrict__ status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    constexpr int H = P / 2;
    static_assert(P <= 2 * kWarps && P <= 32, "at most two stencil rows per warp");
    extern __shared__ float4 smem4[];
    float* tile = reinterpret_cast<float*>(smem4);
    constexpr int PA = (P + 3) & ~3;              // weight rows padded to 16 bytes
    __shared__ __align__(16) float W[kChunk][3][PA];
    __shared__ int B[kChunk][3];
    __shared__ int2 R[kChunk];                    // (tile offset of the stencil corner or -1, its y)
    __shared__ float4 sp[kChunk];
    __shared__ int rs[kMaxRows], pre[kMaxRows + 1];
    __shared__ double red[kWarps];
    __shared__ int is_last;

    const int Tx = g.tg.T[0], Ty = g.tg.T[1], Tz = g.tg.T[2];
    const int TT = Tx * Ty * Tz;
    const int TXY = Tx * Ty;
    const int PS = g.tg.ps;                       // plane stride in shared memory (>= TXY, bank-conflict free)
    const BlockGeom bg = block_geom(g, blockIdx.x);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        float4* t4 = smem4;
        for (int t = threadIdx.x; t < ((PS * Tz) >> 2); t += kThreads) t4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int natoms = block_rows(g, bg, cell_start, rs, pre);   // contains a barrier

    for (int c0 = 0; c0 < natoms; c0 += kChunk) {
        const int nch = min(kChunk, natoms - c0);
        // phase 1: stage the chunk's positions, then per-atom 1D weights (q folded
        // into the x weights) and tile base
        for (int a = threadIdx.x; a < nch; a += kThreads) {
            const int s = block_atom(c0 + a, rs, pre);
            sp[a] = USR_IN_BOUNDS(s, g.max_atoms, status) ? pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nch * 3 * P; idx += kThreads) {
            const int a = idx / (3 * P), rem = idx - a * 3 * P;
            const int ax = rem / P, k = rem - ax * P;
            const float4 p = sp[a];
            // per-axis constants selected without dynamic indexing (keeps them in registers)
            const float pc = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
            const float gs = ax == 0 ? g.box.gs[0] : (ax == 1 ? g.box.gs[1] : g.box.gs[2]);
            const float hh = ax == 0 ? g.hh[0] : (ax == 1 ? g.hh[1] : g.hh[2]);
            const int org = ax == 0 ? bg.o[0] : (ax == 1 ? bg.o[1] : bg.o[2]);
            const int Ta = ax == 0 ? Tx : (ax == 1 ? Ty : Tz);
            const float u = pc * gs;
            const float f = floorf(u);
            const float t = u - f;
            const float d = (float)(k - H + 1) - t;
            float w = __expf(-d * d * hh);
            if (ax == 0) w *= p.w;
            W[a][ax][k] = w;
            if (k == 0) {
                const int base = (int)f - H + 1 - org;
                const bool ok = base >= 0 && base + P <= Ta;
                B[a][ax] = ok ? base : -1;
                if (!ok) atomicOr(status, 2);    // cannot happen for wrapped positions
            }
        }
        __syncthreads();
        // phase 1b: one record per atom, the tile offset of its stencil corner (or -1) and its y
        for (int a = threadIdx.x; a < nch; a += kThreads) {
            const int bx = B[a][0], by = B[a][1], bz = B[a][2];
            R[a] = make_int2(bx < 0 || by < 0 || bz < 0 ? -1 : bz * PS + by * Tx + bx, by);
        }
        __syncthreads();
        // phase 2: warp w owns the tile rows ty = w (mod 8); for each atom it adds
        // the stencil columns of its one or two rows.  Lane = (column jx, group of
        // planes): P columns x G groups, each lane updating PG consecutive planes.
        {
            constexpr int G = 32 / P;                  // plane groups per row
            constexpr int PG = (P + G - 1) / G;        // planes per lane
            static_assert((kWarps & (kWarps - 1)) == 0, "row ownership by a mask");
            const int jx = lane % P, grp = lane / P;
            const int k0 = grp * PG;
            float* const tl = tile + k0 * PS + jx;
            for (int a = 0; a < nch; ++a) {
                const int2 r = R[a];
                if (r.x < 0 || grp >= G) continue;
                float wz[PG];
                #pragma unroll
                for (int k = 0; k < PG; ++k) wz[k] = (k0 + k < P) ? W[a][2][k0 + k] : 0.f;
                const float wxa = W[a][0][jx];
                for (int jy = (warp - r.y) & (kWarps - 1); jy < P; jy += kWarps) {
                    const float v = wxa * W[a][1][jy];
                    float* col = tl + r.x + jy * Tx;
                    float t[PG];
                    #pragma unroll
                    for (int k = 0; k < PG; ++k)
                        if (k0 + k < P) t[k] = col[k * PS];
                    #pragma unroll
                    for (int k = 0; k < PG; ++k)
                        if (k0 + k < P) col[k * PS] = fmaf(v, wz[k], t[k]);
                }
            }
        }
        __syncthreads();
    }

    // store the tile, sum it in a fixed order
    double local;
    {
        const float4* t4 = smem4;
        float4* out4 = reinterpret_cast<float4*>(tilebuf + (size_t)blockIdx.x * TT);
        CSum cs;
        const int pq = TXY >> 2;                  // float4s per plane (TXY is a multiple of 4)
        for (int t = threadIdx.x; t < (TT >> 2); t += kThreads) {
            const int z = t / pq;
            const float4 v = t4[z * (PS >> 2) + (t - z * pq)];   // dense in the tile buffer
            out4[t] = v;
            cs.add(v.x);
            cs.add(v.y);
            cs.add(v.z);
            cs.add(v.w);
        }
        local = warp_sum_c(cs);
    }
    if (lane == 0) red[warp] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w];
        partial[blockIdx.x] = s;
        __threadfence();
        const unsigned int ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        // grid mean from the block sums, in block order (the same whichever CTA is last)
        __threadfence();
        double s = 0.0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += kThreads) s += ((volatile double*)partial)[k];
        s = warp_sum_d(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < kWarps; ++w) tot += red[w];
            *mean = tot / ((double)g.box.n[0] * g.box.n[1] * g.box.n[2]);
            *counter = 0u;
        }
    }
}

/*
 * rho_g = (sum of the tiles holding g, in block order) - mean.  SPLIT = 0
 * writes FP32 rho; 1 and 2 write the operand split of the tensor-core
 * convolution instead: rho = hi + lo with hi rounded to TF32 (1) or BF16 (2).
 */
template <int SPLIT>
__global__ void __launch_bounds__(256) k_tile_reduce(GridArgs g, const float* __restrict__ tilebuf,
                                                     const double* __restrict__ mean, void* __restrict__ rho,
                                                     void* __restrict__ rho_lo, float* __restrict__ rho32,
                                                     int* __restrict__ status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    // grid: x over the (y, x) plane in blocks of 256, y over z (32-bit index arithmetic)
    const int n0 = g.box.n[0], n1 = g.box.n[1];
    const int pxy = blockIdx.x * blockDim.x + threadIdx.x;
    if (pxy >= n0 * n1) return;
    const int y = pxy / n0, x = pxy - y * n0, z = blockIdx.y;
    const long long idx = (long long)z * n0 * n1 + pxy;
    const int T0 = g.tg.T[0], T1 = g.tg.T[1], T2 = g.tg.T[2];
    const long long TT = (long long)T0 * T1 * T2;
    const int nb0 = g.tg.nbk[0], nb1 = g.tg.nbk[1];
    const int cz = g.tab.red_cnt[2][z], cy = g.tab.red_cnt[1][y], cx = g.tab.red_cnt[0][x];
    const int2* pz = g.tab.red_pair[2] + (size_t)z * g.tg.rmax[2];
    const int2* py = g.tab.red_pair[1] + (size_t)y * g.tg.rmax[1];
    const int2* px = g.tab.red_pair[0] + (size_t)x * g.tg.rmax[0];
    float s = 0.f;
    for (int iz = 0; iz < cz; ++iz) {
        const int2 bz = pz[iz];
        for (int iy = 0; iy < cy; ++iy) {
            const int2 by = py[iy];
            const long long rowbase = ((long long)(bz.x * nb1 + by.x) * nb0) * TT + ((long long)bz.y * T1 + by.y) * T0;
            for (int ix = 0; ix < cx; ++ix) {
                const int2 bx = px[ix];
                const long long t = rowbase + (long long)bx.x * TT + bx.y;
                if (USR_IN_BOUNDS(t, (long long)nb0 * nb1 * g.tg.nbk[2] * TT, status)) s += __ldg(tilebuf + t);
            }
        }
    }
    const float v = s - (float)*mean;
    if (SPLIT != 0 && rho32) rho32[idx] = v;     // FP32 copy for the virial convolutions
    if (SPLIT == 0) {
        static_cast<float*>(rho)[idx] = v;
    } else if (SPLIT == 1) {
        uint32_t hb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
        const float h = __uint_as_float(hb);
        static_cast<float*>(rho)[idx] = h;
        static_cast<float*>(rho_lo)[idx] = v - h;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        static_cast<__nv_bfloat16*>(rho)[idx] = h;
        static_cast<__nv_bfloat16*>(rho_lo)[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

/*
 * Grid mean of psi.  Exact arithmetic gives psi no k = 0 mode (rho has its
 * mean removed and the kernels are convolutions), but the FP32 rounding of
 * rho's mean removal leaves a tiny mean that the wide Gaussian terms amplify
 * by their k = 0 transform; the gather subtracts the mean measured here.
 * Fixed-order FP64 partial sums, the last CTA finishes.
 */
__global__ void __launch_bounds__(256) k_grid_mean(long long G, const float* __restrict__ psi,
                                                   const float* __restrict__ w, double scale,
                                                   double* __restrict__ partial, unsigned int* __restrict__ counter,
                                                   double* __restrict__ mean)
{
    __shared__ double red[8];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    CSum cs;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
        if (w)
            cs.add_product(psi[i], w[i]);
        else
            cs.add(psi[i]);
    double s = warp_sum_c(cs);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        partial[blockIdx.x] = t;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double t = 0.0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += 256) t += ((volatile double*)partial)[k];
        t = warp_sum_d(t);
        if (lane == 0) red[warp] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0;
            for (int w = 0; w < 8; ++w) u += red[w];
            *mean = u * scale;
            *counter = 0u;
        }
    }
}

/* out = scale * sum_g a_g b_g in FP64, fixed order (the virial's grid dot products). */
void launch_grid_dot(const GridArgs& g, const float* a, const float* b, double scale, double* partial,
                     unsigned int* counter, double* out, cudaStream_t st)
{
    const long long G = (long long)g.box.n[0] * g.box.n[1] * g.box.n[2];
    k_grid_mean<<<kGridMeanBlocks, 256, 0, st>>>(G, a, b, scale, partial, counter, out);
}

/*
 * W = W_near + delta E_far + 1/2 <rho, psi_ab>: near from the pair kernel's per-unit slots (in unit
 * order; the unit count follows from the group totals of the cell list), far from the six grid dot
 * products (already halved) and E_far.
 */
__global__ void k_virial_finalize(const double* __restrict__ near_w, ClusterList L, int ncell, int nsplit,
                                  const double* __restrict__ dots, const double* __restrict__ energy,
                                  double* __restrict__ W)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int units = nsplit * (L.gfull[ncell] + L.gpart[ncell]);
    double wn[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < units; ++w)
        for (int c = 0; c < 6; ++c) wn[c] += near_w[6 * w + c];
    const double ef = energy[2];
    double t[6];
    for (int c = 0; c < 6; ++c) t[c] = wn[c] + dots[c] + (c < 3 ? ef : 0.0);
    const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
    for (int e = 0; e < 9; ++e) W[e] = t[map[e]];
}

void launch_virial_finalize(const double* near_w, const ClusterList& L, int ncell, const double* dots,
                            const double* energy, double* W, cudaStream_t st)
{
    k_virial_finalize<<<1, 32, 0, st>>>(near_w, L, ncell, near_splits(), dots, energy, W);
}

/* ------------------------------------------------------------------ gather */

/* The pair kernel's near part of sorted atom s: four fixed-point sums (2^-32 units) as FP32. */
__device__ __forceinline__ float4 near_part(const unsigned long long* __restrict__ acc, int s)
{
    const ulonglong2* a2 = reinterpret_cast<const ulonglong2*>(acc + 4 * (size_t)s);
    const ulonglong2 u = a2[0], v = a2[1];
    constexpr float k = 2.3283064365386963e-10f;   // 2^-32, exact
    return make_float4(__ll2float_rn((long long)u.x) * k, __ll2float_rn((long long)u.y) * k,
                       __ll2float_rn((long long)v.x) * k, __ll2float_rn((long long)v.y) * k);
}

/*
 * Far part at every sorted atom (the gather of Sec. V: the spreading Gaussian of the atom against psi,
 * and its gradient), read straight from psi in global memory: consecutive sorted atoms are neighbours in
 * space, so a CTA's stencils overlap and hit in L1 / L2.  A CTA takes consecutive atoms, gather_lanes(P)
 * lanes per atom: lane u takes the stencil columns x = u, u + lanes, ... of every row, contracting z first,
 * so the lanes of an atom read one contiguous run of a row per load.  Writes far4[s] = (-q grad phi, phi
 * before the k = 0 correction); the CTAs also sum psi, and the last one writes its mean.
 */
#ifndef USR_GATHER_MINB
#define USR_GATHER_MINB 2   // CTAs per SM the 8- and 10-point gathers are compiled for (3 spills; measured slower)
#endif
constexpr int kGThreads = USR_GATHER_THREADS;   // gather CTA size
constexpr int kGWarps = kGThreads / 32;
#ifndef USR_GATHER_LANES
#define USR_GATHER_LANES 0   // lanes per atom; 0: 5 for P = 10 (two columns each), else 4
#endif
__host__ __device__ constexpr int gather_lanes(int P)
{
    return USR_GATHER_LANES ? USR_GATHER_LANES : (P == 10 ? 5 : 4);
}

template <int P>
__global__ void __launch_bounds__(kGThreads, (P <= 10 ? USR_GATHER_MINB : 2) * 256 / kGThreads)
    k_gather(const float4* __restrict__ pos, int n, const float* __restrict__ psi, GridArgs g,
             float4* __restrict__ far4, double* __restrict__ partial, unsigned int* __restrict__ counter,
             double* __restrict__ psi_mean, int* __restrict__ status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    constexpr int H = P / 2;
    constexpr int LPA = gather_lanes(P);       // lanes per atom
    constexpr int NC = (P + LPA - 1) / LPA;    // stencil columns per lane
    constexpr int APW = 32 / LPA;              // atoms per warp pass
    constexpr int APC = kGWarps * APW;         // atoms per CTA pass
    __shared__ double red[kGWarps];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = lane / LPA, u = lane % LPA;
    const int n0 = g.box.n[0], n1 = g.box.n[1], n2 = g.box.n[2];
    const long long plane = (long long)n0 * n1;
    // psi's mean (its rounding-level k = 0 mode): this CTA's share of the grid sum first
    CSum ps;
    const long long G = plane * n2;
    for (long long i = (long long)blockIdx.x * kGThreads + threadIdx.x; i < G; i += (long long)gridDim.x * kGThreads)
        ps.add(psi[i]);
    for (int s0 = blockIdx.x * APC + warp * APW; s0 < n; s0 += gridDim.x * APC) {
        const int s = s0 + slot;
        const bool have = slot < APW && s < n;     // lanes past APW x LPA hold no atom
        const float4 p = pos[have ? s : s0];
        const float pc[3] = {p.x, p.y, p.z};
        int base[3];
        float tt[3];
        #pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float uu = pc[a] * g.box.gs[a];
            const float f = floorf(uu);
            tt[a] = uu - f;
            base[a] = (int)f - H + 1;
        }
        float wz[P], dz[P], wx[NC], dx[NC];
        int zi[P], xo[NC];
        #pragma unroll
        for (int k = 0; k < P; ++k) {
            const float d2 = (float)(k - H + 1) - tt[2];
            wz[k] = __expf(-d2 * d2 * g.hh[2]);
            dz[k] = wz[k] * d2 * g.dfac[2];
            zi[k] = wrap_once(base[2] + k, n2);
        }
        #pragma unroll
        for (int m = 0; m < NC; ++m) {
            const int c = u + LPA * m;
            const float d0 = (float)(c - H + 1) - tt[0];
            wx[m] = c < P ? __expf(-d0 * d0 * g.hh[0]) : 0.f;
            dx[m] = wx[m] * d0 * g.dfac[0];
            xo[m] = wrap_once(base[0] + (c < P ? c : 0), n0);
        }
        float aphi = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
        #pragma unroll
        for (int jy = 0; jy < P; ++jy) {
            const float d1 = (float)(jy - H + 1) - tt[1];
            const float wy = __expf(-d1 * d1 * g.hh[1]);
            const float dy = wy * d1 * g.dfac[1];
            const int yo = wrap_once(base[1] + jy, n1) * n0;
            float r0 = 0.f, r1 = 0.f, r2 = 0.f;
            #pragma unroll
            for (int m = 0; m < NC; ++m) {
                if (u + LPA * m >= P) continue;
                const float* col = psi + yo + xo[m];
                float v[P];
                #pragma unroll
                for (int k = 0; k < P; ++k) v[k] = __ldg(col + (long long)zi[k] * plane);
                float c0a = 0.f, c0b = 0.f, c1a = 0.f, c1b = 0.f;
                #pragma unroll
                for (int k = 0; k < P; k += 2) {
                    c0a = fmaf(wz[k], v[k], c0a);
                    c1a = fmaf(dz[k], v[k], c1a);
                    c0b = fmaf(wz[k + 1], v[k + 1], c0b);
                    c1b = fmaf(dz[k + 1], v[k + 1], c1b);
                }
                const float cz0 = c0a + c0b, cz1 = c1a + c1b;
                r0 = fmaf(wx[m], cz0, r0);
                r1 = fmaf(dx[m], cz0, r1);
                r2 = fmaf(wx[m], cz1, r2);
            }
            aphi = fmaf(wy, r0, aphi);
            ax = fmaf(wy, r1, ax);
            ay = fmaf(dy, r0, ay);
            az = fmaf(wy, r2, az);
        }
        // the lanes of an atom hold disjoint partial sums: a butterfly for a power of two, else lane u = 0
        // adds those of u = 1, 2, ... in order
        if ((LPA & (LPA - 1)) == 0) {
            #pragma unroll
            for (int o = 1; o < LPA; o <<= 1) {
                aphi += __shfl_xor_sync(0xffffffffu, aphi, o);
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
                az += __shfl_xor_sync(0xffffffffu, az, o);
            }
        } else {
            const float p0 = aphi, p1 = ax, p2 = ay, p3 = az;
            #pragma unroll
            for (int o = 1; o < LPA; ++o) {
                aphi += __shfl_down_sync(0xffffffffu, p0, o);
                ax += __shfl_down_sync(0xffffffffu, p1, o);
                ay += __shfl_down_sync(0xffffffffu, p2, o);
                az += __shfl_down_sync(0xffffffffu, p3, o);
            }
        }
        if (have && u == 0 && USR_IN_BOUNDS(s, g.max_atoms, status)) {
            const float qi = p.w;
            far4[s] = make_float4(-qi * ax, -qi * ay, -qi * az, aphi);
        }
    }
    // psi's grid sum over all CTAs in a fixed order (the last CTA), then its mean
    const double t = warp_sum_c(ps);
    if (lane == 0) red[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < kGWarps; ++w) v += red[w];
        partial[blockIdx.x] = v;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double a = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kGThreads) a += ((volatile double*)partial)[k];
    a = warp_sum_d(a);
    __syncthreads();
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < kGWarps; ++w) v += red[w];
        *psi_mean = v / (double)G;
        *counter = 0u;
    }
}

/*
 * After the pair kernel and the far gather: per sorted atom s, the result in caller order,
 *   out[perm[s]] = (F_near + F_far, phi_near + phi_far - F(0) q),
 * and the energies E = E_near + E_far + E_self (1/2 sum q phi over Eq. 20's near part, over the grid part,
 * and the self term -1/2 F(0) sum q^2), plus the net charge sum q (a diagnostic: the k = 0 term that a
 * non-zero net charge would carry is the one Eq. 4 drops).  Each block forms the four sums of its atoms;
 * the last block reduces them in block order.
 */
__global__ void __launch_bounds__(kThreads) k_combine(int n, const float4* __restrict__ pos,
                                                      const int* __restrict__ perm,
                                                      const unsigned long long* __restrict__ near_acc,
                                                      const float4* __restrict__ far4, float F0, double F0d,
                                                      float wsum, const double* __restrict__ psi_mean,
                                                      float4* __restrict__ out, float4* __restrict__ near_dbg,
                                                      float4* __restrict__ far_dbg, double* __restrict__ partial,
                                                      unsigned int* __restrict__ counter,
                                                      double* __restrict__ energy,
                                                      double* __restrict__ net_charge, int max_atoms,
                                                      int* __restrict__ status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    __shared__ double red[kWarps][4];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float phi_dc = (float)(*psi_mean) * wsum;   // potential of psi's rounding-level k = 0 mode
    CSum qn, qf, qq, qs;                              // sums of q phi_near, q phi_far, q^2, q
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < n; s += gridDim.x * kThreads) {
        const float4 nr = near_part(near_acc, s), f = far4[s];
        const float qi = pos[s].w;
        const float phi_far = f.w - phi_dc;
        const int i = perm[s];
        qn.add_product(qi, nr.w);
        qf.add_product(qi, phi_far);
        qq.add_product(qi, qi);
        qs.add(qi);
        if (!USR_IN_BOUNDS(i, max_atoms, status)) continue;
        out[i] = make_float4(nr.x + f.x, nr.y + f.y, nr.z + f.z, nr.w + phi_far - F0 * qi);
        if (near_dbg) near_dbg[i] = nr;
        if (far_dbg) far_dbg[i] = make_float4(f.x, f.y, f.z, phi_far);
    }
    double e[4] = {0.5 * warp_sum_c(qn), 0.5 * warp_sum_c(qf), -0.5 * F0d * warp_sum_c(qq), warp_sum_c(qs)};
    if (lane == 0)
        for (int c = 0; c < 4; ++c) red[warp][c] = e[c];
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < kWarps; ++w) v += red[w][threadIdx.x];
        partial[(size_t)blockIdx.x * 4 + threadIdx.x] = v;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    // the last CTA: the four sums over all CTAs in a fixed order
    __threadfence();
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kThreads)
        for (int c = 0; c < 4; ++c) acc[c] += ((volatile double*)partial)[(size_t)k * 4 + c];
    for (int c = 0; c < 4; ++c) acc[c] = warp_sum_d(acc[c]);
    __syncthreads();
    if (lane == 0)
        for (int c = 0; c < 4; ++c) red[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kWarps; ++w)
            for (int c = 0; c < 4; ++c) v[c] += red[w][c];
        energy[0] = v[0] + v[1] + v[2];
        energy[1] = v[0];
        energy[2] = v[1];
        energy[3] = v[2];
        *net_charge = v[3];
        *counter = 0u;
    }
}

/* ------------------------------------------------------------------ launch */

int tile_blocks(const TileGeom& tg) { return tg.nbk[0] * tg.nbk[1] * tg.nbk[2]; }

size_t tile_floats(const TileGeom& tg) { return (size_t)tg.T[0] * tg.T[1] * tg.T[2]; }

template <int P>
static void set_smem(size_t bytes)
{
    cudaFuncSetAttribute(k_spread<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

/* Allow every stencil variant the largest tile a plan may choose. */
usr_status grid_kernel_setup(size_t bytes)
{
    set_smem<8>(bytes);
    set_smem<10>(bytes);
    set_smem<12>(bytes);
    set_smem<14>(bytes);
    set_smem<16>(bytes);
    return cudaGetLastError() == cudaSuccess ? USR_OK : USR_ERR_CUDA;
}

#define USR_SPREAD_CASE(PP)                                                                                     \
    case PP:                                                                                                    \
        launch_pdl(k_spread<PP>, nb, kThreads, smem, st, spos, cell_start, g, tilebuf, partial, counter, mean, \
                   status);                                                                                     \
        break;

void launch_spread(int P, const float4* spos, const int* cell_start, const GridArgs& g, float* tilebuf, int split,
                   void* rho, void* rho_lo, double* partial, unsigned int* counter, double* mean, int* status,
                   cudaStream_t st, float* rho32)
{
    const int nb = tile_blocks(g.tg);
    const size_t smem = sizeof(float) * (size_t)g.tg.ps * g.tg.T[2];
    switch (P) {
        USR_SPREAD_CASE(8)
        USR_SPREAD_CASE(10)
        USR_SPREAD_CASE(12)
        USR_SPREAD_CASE(14)
        default:
        USR_SPREAD_CASE(16)
    }
    const dim3 nr((unsigned)((g.box.n[0] * g.box.n[1] + 255) / 256), (unsigned)g.box.n[2]);
    if (split == 1)
        launch_pdl(k_tile_reduce<1>, nr, 256, 0, st, g, tilebuf, mean, rho, rho_lo, rho32, status);
    else if (split == 2)
        launch_pdl(k_tile_reduce<2>, nr, 256, 0, st, g, tilebuf, mean, rho, rho_lo, rho32, status);
    else
        launch_pdl(k_tile_reduce<0>, nr, 256, 0, st, g, tilebuf, mean, rho, nullptr, nullptr, status);
}

#define USR_GATHER_CASE(PP)                                                                \
    case PP:                                                                               \
        launch_pdl(k_gather<PP>, nb, kGThreads, 0, st, spos, n, psi, g, far4, partial, counter, psi_mean, status); \
        break;

static int gather_blocks(int n, int P)
{
    const int apc = kGThreads / gather_lanes(P);   // atoms per CTA pass
    return std::max(1, std::min(kGatherBlocks, (n + apc - 1) / apc));
}

void launch_gather(int P, int n, const float4* spos, const float* psi, const GridArgs& g, float4* far4,
                   double* partial, unsigned int* counter, double* psi_mean, int* status, cudaStream_t st)
{
    const int nb = gather_blocks(n, P);
    switch (P) {
        USR_GATHER_CASE(8)
        USR_GATHER_CASE(10)
        USR_GATHER_CASE(12)
        USR_GATHER_CASE(14)
        default:
        USR_GATHER_CASE(16)
    }
}

void launch_combine(int n, const float4* spos, const int* perm, const unsigned long long* near_acc,
                    const float4* far4, const GridArgs& g, float4* out,
                    float4* near_dbg, float4* far_dbg, double* partial, unsigned int* counter, double* energy,
                    double* net_charge, int* status, cudaStream_t st)
{
    const int nb = std::max(1, std::min(kCombineBlocks, (n + kThreads - 1) / kThreads));
    k_combine<<<nb, kThreads, 0, st>>>(n, spos, perm, near_acc, far4, g.F0, g.F0d, g.wsum, g.psi_mean, out,
                                       near_dbg, far_dbg, partial, counter, energy, net_charge, g.max_atoms,
                                       status);
}

}  // namespace usr
