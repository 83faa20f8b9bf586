/*
 * k_grid.cu -- the particle-grid legs of the far part (Sec. V with Gaussian
 * spreading, the GSE scheme named in Sec. IV.A).  Both kernels work on
 * blocks of cells: one CTA owns kb_x x kb_y x kb_z cells of the cell list and
 * a shared-memory tile of grid points that covers the P^3 stencils of all
 * their atoms (core + halo, T_x x T_y x T_z points, periodic wrap applied
 * when the tile meets global memory).
 *
 *   spread   rho_g = sum_i q_i exp(-|g - r_i|^2 / (2 sigma_s^2)) (normalisation is
 *            folded into the convolution scale).  One warp per atom adds its
 *            full stencil into the tile with shared-memory atomics; the tile is
 *            then added to the global grid with vector reductions (float4 where
 *            the x rows are 16-byte aligned).  Each CTA also reports the sum of
 *            its tile; the last CTA forms the grid mean (the k = 0 mode,
 *            dropped per Eq. 4).
 *   gather   phi_far,i = sum_g w(g - r_i) psi_g and F_far,i = -q_i grad phi_far,i
 *            (the second spreading Gaussian of Eq. 32's 1/|S(k)|^2).  The CTA
 *            stages its psi tile in shared memory; one warp per atom contracts
 *            the stencil separably (z first, per (x, y) column), adds the near
 *            part and the self term -F(0) q_i, writes (F, phi) in caller order
 *            and reduces E = 1/2 sum q_i phi_i and its parts in FP64.
 */
#include "usr_internal.h"

namespace usr {

namespace {

__device__ __forceinline__ double warp_sum_d(double v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int wrap_mod(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

/* Cell block of this CTA and its tile origin (grid index of tile point 0). */
struct BlockGeom {
    int c0[3], c1[3];   // cell range [c0, c1) per axis
    int o[3];           // tile origin per axis
};

__device__ __forceinline__ BlockGeom block_geom(const GridArgs& g, const TileGeom& tg, int bid, int H, bool align4)
{
    BlockGeom b;
    const int bx = bid % tg.nbk[0], by = (bid / tg.nbk[0]) % tg.nbk[1], bz = bid / (tg.nbk[0] * tg.nbk[1]);
    const int bc[3] = {bx, by, bz};
    #pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.c0[a] = bc[a] * tg.kb[a];
        b.c1[a] = min(g.box.nc[a], b.c0[a] + tg.kb[a]);
        int o = (int)floorf((float)b.c0[a] * tg.wg[a]) - H - 1;
        if (a == 0 && align4) o = o - (((o % 4) + 4) % 4);
        b.o[a] = o;
    }
    return b;
}

}  // namespace

template <int P, bool VEC>
__global__ void __launch_bounds__(256) k_spread(const float4* __restrict__ pos, const int* __restrict__ cell_start,
                                                GridArgs g, TileGeom tg, float* __restrict__ rho,
                                                double* __restrict__ partial, unsigned int* __restrict__ counter,
                                                double* __restrict__ mean, int* __restrict__ status)
{
    constexpr int H = P / 2;
    extern __shared__ float tile[];
    __shared__ double red[8];
    __shared__ int is_last;
    const int Tx = tg.T[0], Ty = tg.T[1], Tz = tg.T[2];
    const int TT = Tx * Ty * Tz;
    const BlockGeom bg = block_geom(g, tg, blockIdx.x, H, VEC);
    for (int t = threadIdx.x; t < TT; t += 256) tile[t] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncx = g.box.nc[0], ncy = g.box.nc[1];
    // atoms of the block: each x-row of cells is a contiguous range of the sorted array
    for (int cz = bg.c0[2]; cz < bg.c1[2]; ++cz) {
        for (int cy = bg.c0[1]; cy < bg.c1[1]; ++cy) {
            const int row = (cz * ncy + cy) * ncx;
            const int as = cell_start[row + bg.c0[0]], ae = cell_start[row + bg.c1[0]];
            for (int ai = as + warp; ai < ae; ai += 8) {
                const float4 p = pos[ai];
                const float pc[3] = {p.x, p.y, p.z};
                int base[3];
                float t[3];
                bool ok = true;
                #pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float u = pc[a] * g.box.gs[a];
                    const float f = floorf(u);
                    t[a] = u - f;
                    base[a] = (int)f - H + 1 - bg.o[a];
                    ok = ok && base[a] >= 0 && base[a] + P <= tg.T[a];
                }
                if (!ok) {                       // cannot happen for in-box atoms; never write outside the tile
                    if (lane == 0) atomicOr(status, 2);
                    continue;
                }
                // z weights in registers, x/y weights per (x, y) column
                float wz[P];
                #pragma unroll
                for (int k = 0; k < P; ++k) {
                    const float d = (float)(k - H + 1) - t[2];
                    wz[k] = __expf(-d * d * g.hh[2]);
                }
                for (int pb = 0; pb < P * P; pb += 32) {
                    const int pp = pb + lane;
                    if (pp < P * P) {
                        const int jy = pp / P, jx = pp - jy * P;
                        const float dx = (float)(jx - H + 1) - t[0];
                        const float dy = (float)(jy - H + 1) - t[1];
                        const float wxy = p.w * __expf(-(dx * dx * g.hh[0] + dy * dy * g.hh[1]));
                        float* col = tile + ((size_t)base[2] * Ty + (base[1] + jy)) * Tx + (base[0] + jx);
                        #pragma unroll
                        for (int k = 0; k < P; ++k) atomicAdd(col + (size_t)k * Tx * Ty, wxy * wz[k]);
                    }
                }
            }
        }
    }
    __syncthreads();
    // add the tile into the periodic grid
    const int n0 = g.box.n[0], n1 = g.box.n[1], n2 = g.box.n[2];
    double local = 0.0;
    if (VEC) {
        const int Tx4 = Tx >> 2;
        for (int t = threadIdx.x; t < Tx4 * Ty * Tz; t += 256) {
            const int x4 = t % Tx4, y = (t / Tx4) % Ty, z = t / (Tx4 * Ty);
            const float* s = tile + ((size_t)z * Ty + y) * Tx + 4 * x4;
            const float4 v = make_float4(s[0], s[1], s[2], s[3]);
            local += (double)v.x + (double)v.y + (double)v.z + (double)v.w;
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
                const int gx = wrap_mod(bg.o[0] + 4 * x4, n0), gy = wrap_mod(bg.o[1] + y, n1),
                          gz = wrap_mod(bg.o[2] + z, n2);
                atomicAdd(reinterpret_cast<float4*>(rho + ((size_t)gz * n1 + gy) * n0 + gx), v);
            }
        }
    } else {
        for (int t = threadIdx.x; t < TT; t += 256) {
            const int x = t % Tx, y = (t / Tx) % Ty, z = t / (Tx * Ty);
            const float v = tile[t];
            local += (double)v;
            if (v != 0.f) {
                const int gx = wrap_mod(bg.o[0] + x, n0), gy = wrap_mod(bg.o[1] + y, n1), gz = wrap_mod(bg.o[2] + z, n2);
                atomicAdd(rho + ((size_t)gz * n1 + gy) * n0 + gx, v);
            }
        }
    }
    local = warp_sum_d(local);
    if (lane == 0) red[warp] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        partial[blockIdx.x] = s;
        __threadfence();
        const unsigned int ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double s = 0.0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += 256) s += ((volatile double*)partial)[k];
        s = warp_sum_d(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < 8; ++w) tot += red[w];
            *mean = tot / ((double)n0 * n1 * n2);
            *counter = 0u;
        }
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_gather(const float4* __restrict__ pos, const int* __restrict__ cell_start,
                                                const int* __restrict__ perm, const float4* __restrict__ near_out,
                                                const float* __restrict__ psi, GridArgs g, TileGeom tg,
                                                float4* __restrict__ out, float4* __restrict__ near_dbg,
                                                float4* __restrict__ far_dbg, double* __restrict__ partial,
                                                unsigned int* __restrict__ counter, double* __restrict__ energy,
                                                int* __restrict__ status)
{
    constexpr int H = P / 2;
    extern __shared__ float tile[];
    __shared__ double red[8][4];
    __shared__ int is_last;
    const int Tx = tg.T[0], Ty = tg.T[1], Tz = tg.T[2];
    const int n0 = g.box.n[0], n1 = g.box.n[1], n2 = g.box.n[2];
    const BlockGeom bg = block_geom(g, tg, blockIdx.x, H, false);
    for (int t = threadIdx.x; t < Tx * Ty * Tz; t += 256) {
        const int x = t % Tx, y = (t / Tx) % Ty, z = t / (Tx * Ty);
        const int gx = wrap_mod(bg.o[0] + x, n0), gy = wrap_mod(bg.o[1] + y, n1), gz = wrap_mod(bg.o[2] + z, n2);
        tile[t] = __ldg(psi + ((size_t)gz * n1 + gy) * n0 + gx);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncx = g.box.nc[0], ncy = g.box.nc[1];
    double e_tot = 0.0, e_near = 0.0, e_far = 0.0, e_self = 0.0;
    for (int cz = bg.c0[2]; cz < bg.c1[2]; ++cz) {
        for (int cy = bg.c0[1]; cy < bg.c1[1]; ++cy) {
            const int row = (cz * ncy + cy) * ncx;
            const int as = cell_start[row + bg.c0[0]], ae = cell_start[row + bg.c1[0]];
            for (int s = as + warp; s < ae; s += 8) {
                const float4 p = pos[s];
                const float pc[3] = {p.x, p.y, p.z};
                int base[3];
                float t[3];
                bool ok = true;
                #pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float u = pc[a] * g.box.gs[a];
                    const float f = floorf(u);
                    t[a] = u - f;
                    base[a] = (int)f - H + 1 - bg.o[a];
                    ok = ok && base[a] >= 0 && base[a] + P <= tg.T[a];
                }
                float aphi = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
                if (ok) {
                    float wz[P], dz[P];
                    #pragma unroll
                    for (int k = 0; k < P; ++k) {
                        const float d = (float)(k - H + 1) - t[2];
                        wz[k] = __expf(-d * d * g.hh[2]);
                        dz[k] = wz[k] * d * g.dfac[2];
                    }
                    for (int pb = 0; pb < P * P; pb += 32) {
                        const int pp = pb + lane;
                        if (pp < P * P) {
                            const int jy = pp / P, jx = pp - jy * P;
                            const float dx = (float)(jx - H + 1) - t[0];
                            const float dy = (float)(jy - H + 1) - t[1];
                            const float wx = __expf(-dx * dx * g.hh[0]);
                            const float wy = __expf(-dy * dy * g.hh[1]);
                            const float* col = tile + ((size_t)base[2] * Ty + (base[1] + jy)) * Tx + (base[0] + jx);
                            float cz0 = 0.f, cz1 = 0.f;
                            #pragma unroll
                            for (int k = 0; k < P; ++k) {
                                const float v = col[(size_t)k * Tx * Ty];
                                cz0 = fmaf(wz[k], v, cz0);
                                cz1 = fmaf(dz[k], v, cz1);
                            }
                            const float wxy = wx * wy;
                            aphi = fmaf(wxy, cz0, aphi);
                            ax = fmaf(wx * dx * g.dfac[0] * wy, cz0, ax);
                            ay = fmaf(wx * wy * dy * g.dfac[1], cz0, ay);
                            az = fmaf(wxy, cz1, az);
                        }
                    }
                } else if (lane == 0) {
                    atomicOr(status, 2);
                }
                aphi = warp_sum_f(aphi);
                ax = warp_sum_f(ax);
                ay = warp_sum_f(ay);
                az = warp_sum_f(az);
                if (lane == 0) {
                    const int i = perm[s];
                    const float qi = p.w;
                    const float4 nr = near_out[s];
                    const float fx = -qi * ax, fy = -qi * ay, fz = -qi * az;
                    const float phi = nr.w + aphi - g.F0 * qi;
                    out[i] = make_float4(nr.x + fx, nr.y + fy, nr.z + fz, phi);
                    if (near_dbg) near_dbg[i] = nr;
                    if (far_dbg) far_dbg[i] = make_float4(fx, fy, fz, aphi);
                    const double en = 0.5 * (double)qi * (double)nr.w;
                    const double ef = 0.5 * (double)qi * (double)aphi;
                    const double es = -0.5 * (double)g.F0 * (double)qi * (double)qi;
                    e_near += en;
                    e_far += ef;
                    e_self += es;
                    e_tot += en + ef + es;
                }
            }
        }
    }
    if (lane == 0) {
        red[warp][0] = e_tot;
        red[warp][1] = e_near;
        red[warp][2] = e_far;
        red[warp][3] = e_self;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        partial[(size_t)blockIdx.x * 4 + threadIdx.x] = v;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = threadIdx.x; k < (int)gridDim.x; k += 256) {
            #pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += ((volatile double*)partial)[(size_t)k * 4 + c];
        }
        #pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = warp_sum_d(acc[c]);
        __syncthreads();
        if (lane == 0)
            for (int c = 0; c < 4; ++c) red[warp][c] = acc[c];
        __syncthreads();
        if (threadIdx.x < 4) {
            double v = 0.0;
            for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
            energy[threadIdx.x] = v;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

int tile_blocks(const TileGeom& tg) { return tg.nbk[0] * tg.nbk[1] * tg.nbk[2]; }

size_t tile_bytes(const TileGeom& tg) { return sizeof(float) * (size_t)tg.T[0] * tg.T[1] * tg.T[2]; }

template <int P>
static void set_smem(size_t bytes)
{
    cudaFuncSetAttribute(k_spread<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_spread<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_gather<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

usr_status grid_kernel_setup(int P, size_t bytes)
{
    switch (P) {
        case 8: set_smem<8>(bytes); break;
        case 10: set_smem<10>(bytes); break;
        case 12: set_smem<12>(bytes); break;
        case 14: set_smem<14>(bytes); break;
        default: set_smem<16>(bytes); break;
    }
    return cudaGetLastError() == cudaSuccess ? USR_OK : USR_ERR_CUDA;
}

#define USR_SPREAD_CASE(PP)                                                                                         \
    case PP:                                                                                                        \
        if (vec)                                                                                                    \
            k_spread<PP, true><<<nb, 256, smem, st>>>(spos, cell_start, g, tg, rho, partial, counter, mean, status); \
        else                                                                                                        \
            k_spread<PP, false><<<nb, 256, smem, st>>>(spos, cell_start, g, tg, rho, partial, counter, mean, status); \
        break;

void launch_spread(int P, bool vec, const float4* spos, const int* cell_start, const GridArgs& g, const TileGeom& tg,
                   float* rho, double* partial, unsigned int* counter, double* mean, int* status, cudaStream_t st)
{
    const int nb = tile_blocks(tg);
    const size_t smem = tile_bytes(tg);
    const long long G = (long long)g.box.n[0] * g.box.n[1] * g.box.n[2];
    cudaMemsetAsync(rho, 0, sizeof(float) * (size_t)G, st);
    switch (P) {
        USR_SPREAD_CASE(8)
        USR_SPREAD_CASE(10)
        USR_SPREAD_CASE(12)
        USR_SPREAD_CASE(14)
        default:
        USR_SPREAD_CASE(16)
    }
}

#define USR_GATHER_CASE(PP)                                                                                     \
    case PP:                                                                                                    \
        k_gather<PP><<<nb, 256, smem, st>>>(spos, cell_start, perm, near_out, psi, g, tg, out, near_dbg, far_dbg, \
                                             partial, counter, energy, status);                                 \
        break;

void launch_gather(int P, const float4* spos, const int* cell_start, const int* perm, const float4* near_out,
                   const float* psi, const GridArgs& g, const TileGeom& tg, float4* out, float4* near_dbg,
                   float4* far_dbg, double* partial, unsigned int* counter, double* energy, int* status,
                   cudaStream_t st)
{
    const int nb = tile_blocks(tg);
    const size_t smem = tile_bytes(tg);
    switch (P) {
        USR_GATHER_CASE(8)
        USR_GATHER_CASE(10)
        USR_GATHER_CASE(12)
        USR_GATHER_CASE(14)
        default:
        USR_GATHER_CASE(16)
    }
}

}  // namespace usr
