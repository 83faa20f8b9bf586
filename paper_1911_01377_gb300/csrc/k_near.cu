/*
 * k_near.cu -- near part of the u-series, Eq. 20:
 *   N(r) = 1/r - F(r) for r < r_c, 0 otherwise
 *   phi_i^near = sum_j q_j N(r_ij),   F_i^near = q_i sum_j q_j (1/r^3 + F'(r)/r) (r_i - r_j)
 * over all j != i and periodic images.
 *
 * One CTA per home cell; each thread owns one home atom.  The 27 neighbour
 * cells (edge >= r_c, >= 3 per axis, so every image appears once) are staged
 * through shared memory as float4 tiles with their periodic shift already
 * added, so the inner loop is broadcast smem reads and FP32 math:
 *   r^2 by the single-precision pair predicate (fmaf(dz,dz,fmaf(dy,dy,dx*dx)))
 *   1/r by rsqrt plus one Newton step
 *   F(u = r^2) = sum of the explicit narrow Gaussians + a polynomial in
 *   s = 2u/r_c^2 - 1 (Horner, value and derivative together)
 * Every pair is evaluated from both ends, so there are no atomics and each
 * output is written once.
 */
#include "usr_internal.h"

namespace usr {

template <int DEG, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_near(const float4* __restrict__ pos, const int* __restrict__ cell_start,
                                                NearArgs a, float4* __restrict__ out)
{
    __shared__ float4 sj[BLOCK];
    const int c = blockIdx.x;
    const int ncx = a.box.nc[0], ncy = a.box.nc[1], ncz = a.box.nc[2];
    const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
    const int hs = cell_start[c], he = cell_start[c + 1];
    for (int base = hs; base < he; base += BLOCK) {
        const int i = base + threadIdx.x;
        const bool act = i < he;
        const float4 pi = act ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float fx = 0.f, fy = 0.f, fz = 0.f, ph = 0.f;
        for (int nb = 0; nb < 27; ++nb) {
            int ox = nb % 3 - 1, oy = (nb / 3) % 3 - 1, oz = nb / 9 - 1;
            int nx = cx + ox, ny = cy + oy, nz = cz + oz;
            float sx = 0.f, sy = 0.f, sz = 0.f;
            if (nx < 0) { nx += ncx; sx = -a.box.L[0]; } else if (nx >= ncx) { nx -= ncx; sx = a.box.L[0]; }
            if (ny < 0) { ny += ncy; sy = -a.box.L[1]; } else if (ny >= ncy) { ny -= ncy; sy = a.box.L[1]; }
            if (nz < 0) { nz += ncz; sz = -a.box.L[2]; } else if (nz >= ncz) { nz -= ncz; sz = a.box.L[2]; }
            const int ncell = (nz * ncy + ny) * ncx + nx;
            const int js = cell_start[ncell], je = cell_start[ncell + 1];
            for (int jb = js; jb < je; jb += BLOCK) {
                __syncthreads();
                if (jb + (int)threadIdx.x < je) {
                    float4 p = pos[jb + threadIdx.x];
                    p.x = __fadd_rn(p.x, sx);
                    p.y = __fadd_rn(p.y, sy);
                    p.z = __fadd_rn(p.z, sz);
                    sj[threadIdx.x] = p;
                }
                __syncthreads();
                const int cnt = min(BLOCK, je - jb);
                if (act) {
                    for (int k = 0; k < cnt; ++k) {
                        const float4 pj = sj[k];
                        const float dx = __fsub_rn(pi.x, pj.x);
                        const float dy = __fsub_rn(pi.y, pj.y);
                        const float dz = __fsub_rn(pi.z, pj.z);
                        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                        if (r2 < a.rc2 && jb + k != i) {
                            float ri = rsqrtf(r2);
                            ri = ri * fmaf(-0.5f * r2 * ri, ri, 1.5f);
                            const float s = fmaf(r2, a.two_over_rc2, -1.0f);
                            float p = a.poly[DEG], dp = 0.f;
                            #pragma unroll
                            for (int d = DEG - 1; d >= 0; --d) {
                                dp = fmaf(dp, s, p);
                                p = fmaf(p, s, a.poly[d]);
                            }
                            float dFdu = dp * a.two_over_rc2;
                            for (int e = 0; e < a.n_explicit; ++e) {
                                float g = a.ea[e] * expf(-r2 * a.einv[e]);
                                p += g;
                                dFdu = fmaf(-g, a.einv[e], dFdu);
                            }
                            const float qj = pj.w;
                            ph = fmaf(qj, ri - p, ph);
                            const float gsc = qj * fmaf(ri * ri, ri, 2.0f * dFdu);
                            fx = fmaf(gsc, dx, fx);
                            fy = fmaf(gsc, dy, fy);
                            fz = fmaf(gsc, dz, fz);
                        }
                    }
                }
            }
        }
        if (act) out[i] = make_float4(pi.w * fx, pi.w * fy, pi.w * fz, ph);
    }
}

/* Pair-list summary (count and order-free hash of partner caller indices). */
__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(128) k_pairs(const float4* __restrict__ pos, const int* __restrict__ cell_start,
                                               const int* __restrict__ perm, NearArgs a, int* __restrict__ count,
                                               unsigned long long* __restrict__ hash)
{
    __shared__ float4 sj[128];
    __shared__ int sid[128];
    const int c = blockIdx.x;
    const int ncx = a.box.nc[0], ncy = a.box.nc[1], ncz = a.box.nc[2];
    const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
    const int hs = cell_start[c], he = cell_start[c + 1];
    for (int base = hs; base < he; base += 128) {
        const int i = base + threadIdx.x;
        const bool act = i < he;
        const float4 pi = act ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        int cnt_i = 0;
        unsigned long long h = 0;
        for (int nb = 0; nb < 27; ++nb) {
            int ox = nb % 3 - 1, oy = (nb / 3) % 3 - 1, oz = nb / 9 - 1;
            int nx = cx + ox, ny = cy + oy, nz = cz + oz;
            float sx = 0.f, sy = 0.f, sz = 0.f;
            if (nx < 0) { nx += ncx; sx = -a.box.L[0]; } else if (nx >= ncx) { nx -= ncx; sx = a.box.L[0]; }
            if (ny < 0) { ny += ncy; sy = -a.box.L[1]; } else if (ny >= ncy) { ny -= ncy; sy = a.box.L[1]; }
            if (nz < 0) { nz += ncz; sz = -a.box.L[2]; } else if (nz >= ncz) { nz -= ncz; sz = a.box.L[2]; }
            const int ncell = (nz * ncy + ny) * ncx + nx;
            const int js = cell_start[ncell], je = cell_start[ncell + 1];
            for (int jb = js; jb < je; jb += 128) {
                __syncthreads();
                if (jb + (int)threadIdx.x < je) {
                    float4 p = pos[jb + threadIdx.x];
                    p.x = __fadd_rn(p.x, sx);
                    p.y = __fadd_rn(p.y, sy);
                    p.z = __fadd_rn(p.z, sz);
                    sj[threadIdx.x] = p;
                    sid[threadIdx.x] = perm[jb + threadIdx.x];
                }
                __syncthreads();
                const int cnt = min(128, je - jb);
                if (act) {
                    for (int k = 0; k < cnt; ++k) {
                        const float4 pj = sj[k];
                        const float dx = __fsub_rn(pi.x, pj.x);
                        const float dy = __fsub_rn(pi.y, pj.y);
                        const float dz = __fsub_rn(pi.z, pj.z);
                        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                        if (r2 < a.rc2 && jb + k != i) {
                            ++cnt_i;
                            h += mix64((unsigned long long)sid[k]);
                        }
                    }
                }
            }
        }
        if (act) {
            int ci = perm[i];
            count[ci] = cnt_i;
            hash[ci] = h;
        }
    }
}

template <int DEG>
static void launch_near_deg(int ncell, int block, const float4* spos, const int* cell_start, const NearArgs& a,
                            float4* out, cudaStream_t st)
{
    if (block <= 64)
        k_near<DEG, 64><<<ncell, 64, 0, st>>>(spos, cell_start, a, out);
    else
        k_near<DEG, 128><<<ncell, 128, 0, st>>>(spos, cell_start, a, out);
}

void launch_near(int ncell, int block, int deg, const float4* spos, const int* cell_start, const NearArgs& a,
                 float4* out, cudaStream_t st)
{
    switch (deg) {
        case 8: launch_near_deg<8>(ncell, block, spos, cell_start, a, out, st); break;
        case 12: launch_near_deg<12>(ncell, block, spos, cell_start, a, out, st); break;
        case 16: launch_near_deg<16>(ncell, block, spos, cell_start, a, out, st); break;
        case 20: launch_near_deg<20>(ncell, block, spos, cell_start, a, out, st); break;
        default: launch_near_deg<24>(ncell, block, spos, cell_start, a, out, st); break;
    }
}

void launch_pairs(int ncell, const float4* spos, const int* cell_start, const int* perm, const NearArgs& a,
                  int* count, unsigned long long* hash, cudaStream_t st)
{
    k_pairs<<<ncell, 128, 0, st>>>(spos, cell_start, perm, a, count, hash);
}

}  // namespace usr
