/*
 * k_near.cu -- near part of the u-series, Eq. 20:
 *   N(r) = 1/r - F(r) for r < r_c, 0 otherwise
 *   phi_i^near = sum_j q_j N(r_ij),   F_i^near = q_i sum_j q_j (1/r^3 + F'(r)/r) (r_i - r_j)
 * over all j != i and periodic images.
 *
 * Cluster-pair scheme: each cell's atoms come in 8-atom spatial clusters
 * (k_cluster_build).  One warp owns one i-cluster; lanes are (i = lane / 4,
 * j = lane % 4), so a warp step evaluates an 8 x 4 block of pairs with every
 * lane on the same path.  The warp walks the j-clusters of the 27 neighbour
 * cells (edge >= r_c, >= 3 per axis, so every image appears once), tests 32
 * candidate bounding boxes at a time against its own box (a conservative
 * test: it uses the same rounding as the pair distance, so it never drops a
 * pair the single-precision predicate accepts) and runs the surviving
 * cluster pairs as two 8 x 4 steps.  Every pair is evaluated from both ends,
 * so i-forces stay in registers: no atomics, a fixed order, one write per atom.
 *
 * Per pair: r^2 by the single-precision predicate fmaf(dz,dz,fmaf(dy,dy,dx*dx));
 * 1/r by rsqrt plus one Newton step; F(u = r^2) = explicit narrow Gaussians
 * plus a polynomial in s = 2u / r_c^2 - 1 (Horner, value and derivative).
 */
#include "usr_internal.h"

namespace usr {

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * COUNT = true: instead of the interaction, count partners and hash their caller indices.
 * VIR = true: also accumulate the pair virial 1/2 sum d (x) f (six components, FP32 per lane,
 * summed over the warp in a fixed order and written as FP64 to vir[6 * warp ..], one slot per
 * warp of the grid).
 */
template <int DEG, bool COUNT, bool VIR>
__global__ void __launch_bounds__(128) k_near_cl(const float4* __restrict__ cpos, const int* __restrict__ cidx,
                                                 const int* __restrict__ ccell, const float4* __restrict__ bblo,
                                                 const float4* __restrict__ bbhi, const int* __restrict__ pstart,
                                                 const int* __restrict__ perm, NearArgs a, float4* __restrict__ out,
                                                 int* __restrict__ count, unsigned long long* __restrict__ hash,
                                                 double* __restrict__ vir)
{
    const int ncx = a.box.nc[0], ncy = a.box.nc[1], ncz = a.box.nc[2];
    const int ncl = pstart[ncx * ncy * ncz] >> 3;
    const int ic = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    float vxx = 0.f, vyy = 0.f, vzz = 0.f, vxy = 0.f, vxz = 0.f, vyz = 0.f;
    if (ic >= ncl) {
        if (VIR && lane < 6) vir[6 * ic + lane] = 0.0;    // one slot per warp, idle warps write zeros
        return;
    }
    const int il = lane >> 2, jl = lane & 3;
    const int islot = ic * 8 + il;
    const float4 pi = cpos[islot];
    const float4 blo = bblo[ic], bhi = bbhi[ic];
    const int c = ccell[ic];
    const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
    float fx = 0.f, fy = 0.f, fz = 0.f, ph = 0.f;
    int cnt = 0;
    unsigned long long h = 0ull;
    for (int nb = 0; nb < 27; ++nb) {
        int nx = cx + nb % 3 - 1, ny = cy + (nb / 3) % 3 - 1, nz = cz + nb / 9 - 1;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        if (nx < 0) { nx += ncx; sx = -a.box.L[0]; } else if (nx >= ncx) { nx -= ncx; sx = a.box.L[0]; }
        if (ny < 0) { ny += ncy; sy = -a.box.L[1]; } else if (ny >= ncy) { ny -= ncy; sy = a.box.L[1]; }
        if (nz < 0) { nz += ncz; sz = -a.box.L[2]; } else if (nz >= ncz) { nz -= ncz; sz = a.box.L[2]; }
        const int nc = (nz * ncy + ny) * ncx + nx;
        const int jc0 = pstart[nc] >> 3, jc1 = pstart[nc + 1] >> 3;
        for (int jb = jc0; jb < jc1; jb += 32) {
            const int jc = jb + lane;
            bool near = false;
            if (jc < jc1) {
                const float4 lo = bblo[jc], hi = bbhi[jc];
                // gap between the boxes, rounded like a pair distance
                const float gx = fmaxf(0.f, fmaxf(__fsub_rn(__fadd_rn(lo.x, sx), bhi.x), __fsub_rn(blo.x, __fadd_rn(hi.x, sx))));
                const float gy = fmaxf(0.f, fmaxf(__fsub_rn(__fadd_rn(lo.y, sy), bhi.y), __fsub_rn(blo.y, __fadd_rn(hi.y, sy))));
                const float gz = fmaxf(0.f, fmaxf(__fsub_rn(__fadd_rn(lo.z, sz), bhi.z), __fsub_rn(blo.z, __fadd_rn(hi.z, sz))));
                near = __fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx))) < a.rc2;
            }
            unsigned int m = __ballot_sync(0xffffffffu, near);
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                const int jcl = jb + k;
                #pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int jslot = jcl * 8 + half * 4 + jl;
                    const float4 pj = cpos[jslot];
                    const float dx = __fsub_rn(pi.x, __fadd_rn(pj.x, sx));
                    const float dy = __fsub_rn(pi.y, __fadd_rn(pj.y, sy));
                    const float dz = __fsub_rn(pi.z, __fadd_rn(pj.z, sz));
                    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                    const bool in = r2 < a.rc2 && (jslot != islot || nb != 13);
                    if (COUNT) {
                        if (in) {
                            const int sj = cidx[jslot];
                            ++cnt;
                            h += mix64((unsigned long long)perm[sj]);
                        }
                    } else if (in) {
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
                            const float g = a.ea[e] * __expf(-r2 * a.einv[e]);
                            p += g;
                            dFdu = fmaf(-g, a.einv[e], dFdu);
                        }
                        const float qj = pj.w;
                        ph = fmaf(qj, ri - p, ph);
                        const float gsc = qj * fmaf(ri * ri, ri, 2.0f * dFdu);
                        fx = fmaf(gsc, dx, fx);
                        fy = fmaf(gsc, dy, fy);
                        fz = fmaf(gsc, dz, fz);
                        if (VIR) {
                            vxx = fmaf(gsc * dx, dx, vxx);
                            vyy = fmaf(gsc * dy, dy, vyy);
                            vzz = fmaf(gsc * dz, dz, vzz);
                            vxy = fmaf(gsc * dx, dy, vxy);
                            vxz = fmaf(gsc * dx, dz, vxz);
                            vyz = fmaf(gsc * dy, dz, vyz);
                        }
                    }
                }
            }
        }
    }
    // the four lanes of an i-atom hold disjoint partial sums
    #pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
        ph += __shfl_xor_sync(0xffffffffu, ph, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        h += __shfl_xor_sync(0xffffffffu, h, o);
    }
    const int si = cidx[islot];
    if (jl == 0 && si >= 0) {
        if (COUNT) {
            const int ci = perm[si];
            count[ci] = cnt;
            hash[ci] = h;
        } else {
            out[si] = make_float4(pi.w * fx, pi.w * fy, pi.w * fz, ph);
        }
    }
    if (VIR) {
        // 1/2 q_i sum_j gsc d (x) d, summed over the warp (fixed tree), then over the CTA
        const double hq = si >= 0 ? 0.5 * (double)pi.w : 0.0;    // padding rows contribute nothing
        double v[6] = {hq * vxx, hq * vyy, hq * vzz, hq * vxy, hq * vxz, hq * vyz};
        if (si < 0)
            for (int c = 0; c < 6; ++c) v[c] = 0.0;
        #pragma unroll
        for (int c = 0; c < 6; ++c)
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
        if (lane == 0)
            for (int c = 0; c < 6; ++c) vir[6 * ic + c] = v[c];
    }
}

template <int DEG, bool COUNT>
static void launch_cl(int max_clusters, const float4* cpos, const int* cidx, const int* ccell, const float4* bblo,
                      const float4* bbhi, const int* pstart, const int* perm, const NearArgs& a, float4* out,
                      int* count, unsigned long long* hash, cudaStream_t st, double* vir = nullptr)
{
    const int blocks = (max_clusters + 3) / 4;
    if (vir)
        k_near_cl<DEG, COUNT, true><<<blocks, 128, 0, st>>>(cpos, cidx, ccell, bblo, bbhi, pstart, perm, a, out, count,
                                                             hash, vir);
    else
        k_near_cl<DEG, COUNT, false><<<blocks, 128, 0, st>>>(cpos, cidx, ccell, bblo, bbhi, pstart, perm, a, out,
                                                              count, hash, nullptr);
}

int near_warps(int max_clusters) { return 4 * ((max_clusters + 3) / 4); }

void launch_near(int max_clusters, int deg, const float4* cpos, const int* cidx, const int* ccell, const float4* bblo,
                 const float4* bbhi, const int* pstart, const NearArgs& a, float4* out, cudaStream_t st, double* vir)
{
    switch (deg) {
        case 6: launch_cl<6, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
        case 7: launch_cl<7, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
        case 8: launch_cl<8, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
        case 10: launch_cl<10, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
        case 12: launch_cl<12, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
        case 16: launch_cl<16, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
        case 20: launch_cl<20, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
        default: launch_cl<24, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr, nullptr, st, vir); break;
    }
}

void launch_pairs(int max_clusters, const float4* cpos, const int* cidx, const int* ccell, const float4* bblo,
                  const float4* bbhi, const int* pstart, const int* perm, const NearArgs& a, int* count,
                  unsigned long long* hash, cudaStream_t st)
{
    launch_cl<8, true>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, perm, a, nullptr, count, hash, st);
}

}  // namespace usr
