/*
 * k_near.cu -- near part of the u-series, Eq. 20:
 *   N(r) = 1/r - F(r) for r < r_c, 0 otherwise
 *   phi_i^near = sum_j q_j N(r_ij),   F_i^near = q_i sum_j q_j (1/r^3 + F'(r)/r) (r_i - r_j)
 * over all j != i and periodic images.
 *
 * Cluster-pair scheme: each cell's atoms come in 8-atom spatial clusters
 * (k_cell_build).  One warp owns one i-cluster; lane (i = lane / 4, g =
 * lane % 4) takes the j atoms g and g + 4 of each j cluster in two-wide FP32,
 * so a warp step evaluates an 8 x 8 cluster pair with every lane on the same
 * path.  The warp walks the j-clusters of the 27 neighbour cells (edge >= r_c,
 * >= 3 per axis, so every image appears once), tests 32 candidate bounding
 * boxes at a time against its own box (a conservative test: it uses the same
 * rounding as the pair distance, so it never drops a pair the single-precision
 * predicate accepts) and runs one step per surviving cluster pair.  Every pair
 * is evaluated from both ends, so i-forces stay in registers: no atomics, a
 * fixed order, one write per atom.
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
 * Two-wide FP32 arithmetic (add/sub/mul/fma .f32x2): each lane evaluates its
 * two pairs of a cluster pair (j atoms g and g + 4) in one instruction stream,
 * halving the issued instructions of the pair arithmetic.  Each element is
 * rounded exactly as the scalar instruction would round it.
 */
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void upk(f2 r, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float exp2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ f2 dup(float a) { return pk(a, a); }

/*
 * COUNT = true: instead of the interaction, count partners and hash their caller indices.
 * VIR = true: also accumulate the pair virial 1/2 sum d (x) f (six components, FP32 per lane,
 * summed over the warp in a fixed order and written as FP64 to vir[6 * warp ..], one slot per
 * warp of the grid).
 *
 * Lane (il = lane / 4, g = lane % 4) holds i atom il and, for every cluster pair, the two
 * j atoms g and g + 4 of the j cluster (the paired layout of k_cell_build).
 */
template <int DEG, int NEXP, bool COUNT, bool VIR>
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
    f2 vxx = 0ull, vyy = 0ull, vzz = 0ull, vxy = 0ull, vxz = 0ull, vyz = 0ull;
    if (ic >= ncl) {
        if (VIR && lane < 6) vir[6 * ic + lane] = 0.0;    // one slot per warp, idle warps write zeros
        return;
    }
    const int il = lane >> 2, g = lane & 3;
    const int islot = ic * 8 + il;
    const float* cf = reinterpret_cast<const float*>(cpos);
    const int io = ic * 32 + 8 * (il & 3) + (il >> 2);
    const float4 pi = make_float4(cf[io], cf[io + 2], cf[io + 4], cf[io + 6]);
    const f2 pix = dup(pi.x), piy = dup(pi.y), piz = dup(pi.z);
    const float4 blo = bblo[ic], bhi = bbhi[ic];
    const int c = ccell[ic];
    const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
    const ulonglong2* cp2 = reinterpret_cast<const ulonglong2*>(cpos);
    f2 fx = 0ull, fy = 0ull, fz = 0ull, ph = 0ull;
    int cnt = 0;
    unsigned long long h = 0ull;
    const f2 c_two = dup(a.two_over_rc2), c_m1 = dup(-1.0f), c_mh = dup(-0.5f), c_3h = dup(1.5f);
    const f2 c_d2 = dup(2.0f * a.two_over_rc2);
    for (int nb = 0; nb < 27; ++nb) {
        int nx = cx + nb % 3 - 1, ny = cy + (nb / 3) % 3 - 1, nz = cz + nb / 9 - 1;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        if (nx < 0) { nx += ncx; sx = -a.box.L[0]; } else if (nx >= ncx) { nx -= ncx; sx = a.box.L[0]; }
        if (ny < 0) { ny += ncy; sy = -a.box.L[1]; } else if (ny >= ncy) { ny -= ncy; sy = a.box.L[1]; }
        if (nz < 0) { nz += ncz; sz = -a.box.L[2]; } else if (nz >= ncz) { nz -= ncz; sz = a.box.L[2]; }
        const f2 sx2 = dup(sx), sy2 = dup(sy), sz2 = dup(sz);
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
                const ulonglong2 A = cp2[jcl * 8 + 2 * g];         // (x_g, x_g+4), (y_g, y_g+4)
                const ulonglong2 B = cp2[jcl * 8 + 2 * g + 1];     // (z_g, z_g+4), (q_g, q_g+4)
                const f2 dx = sub2(pix, add2(A.x, sx2));
                const f2 dy = sub2(piy, add2(A.y, sy2));
                const f2 dz = sub2(piz, add2(B.x, sz2));
                const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                float r2a, r2b;
                upk(r2, r2a, r2b);
                const bool self = nb == 13 && jcl == ic;
                const bool ina = r2a < a.rc2 && !(self && g == il);
                const bool inb = r2b < a.rc2 && !(self && g + 4 == il);
                if (COUNT) {
                    if (ina) {
                        ++cnt;
                        h += mix64((unsigned long long)perm[cidx[jcl * 8 + g]]);
                    }
                    if (inb) {
                        ++cnt;
                        h += mix64((unsigned long long)perm[cidx[jcl * 8 + 4 + g]]);
                    }
                } else if (ina || inb) {
                    // pairs outside r_c (or the atom itself) get r^2 = r_c^2 and q_j = 0: finite, adds 0
                    float qa, qb;
                    upk(B.y, qa, qb);
                    const f2 u = pk(ina ? r2a : a.rc2, inb ? r2b : a.rc2);
                    const f2 q = pk(ina ? qa : 0.f, inb ? qb : 0.f);
                    float ra, rb;
                    upk(u, ra, rb);
                    f2 ri = pk(rsqrt_ftz(ra), rsqrt_ftz(rb));
                    ri = mul2(ri, fma2(mul2(mul2(u, ri), ri), c_mh, c_3h));    // one Newton step
                    const f2 s = fma2(u, c_two, c_m1);
                    f2 p = dup(a.poly[DEG]), dp = p;
                    p = fma2(p, s, dup(a.poly[DEG - 1]));
                    #pragma unroll
                    for (int d = DEG - 2; d >= 0; --d) {
                        dp = fma2(dp, s, p);
                        p = fma2(p, s, dup(a.poly[d]));
                    }
                    f2 d2 = mul2(dp, c_d2);                                 // 2 dF/du
                    // NEXP >= 0: that many explicit Gaussians, unrolled; -1: a.n_explicit of them
                    const int nexp = NEXP >= 0 ? NEXP : a.n_explicit;
                    #pragma unroll
                    for (int e = 0; e < nexp; ++e) {
                        float ea_, eb_;
                        upk(mul2(u, dup(a.el2[e])), ea_, eb_);
                        const f2 gg = mul2(pk(exp2_ftz(ea_), exp2_ftz(eb_)), dup(a.ea[e]));
                        p = add2(p, gg);
                        d2 = fma2(gg, dup(a.ne2[e]), d2);
                    }
                    ph = fma2(q, sub2(ri, p), ph);
                    const f2 gsc = mul2(q, fma2(mul2(ri, ri), ri, d2));
                    fx = fma2(gsc, dx, fx);
                    fy = fma2(gsc, dy, fy);
                    fz = fma2(gsc, dz, fz);
                    if (VIR) {
                        const f2 gx = mul2(gsc, dx), gy = mul2(gsc, dy);
                        vxx = fma2(gx, dx, vxx);
                        vxy = fma2(gx, dy, vxy);
                        vxz = fma2(gx, dz, vxz);
                        vyy = fma2(gy, dy, vyy);
                        vyz = fma2(gy, dz, vyz);
                        vzz = fma2(mul2(gsc, dz), dz, vzz);
                    }
                }
            }
        }
    }
    float fxs, fys, fzs, phs;
    {
        float u0, u1;
        upk(fx, u0, u1); fxs = u0 + u1;
        upk(fy, u0, u1); fys = u0 + u1;
        upk(fz, u0, u1); fzs = u0 + u1;
        upk(ph, u0, u1); phs = u0 + u1;
    }
    // the four lanes of an i-atom hold disjoint partial sums
    #pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        fxs += __shfl_xor_sync(0xffffffffu, fxs, o);
        fys += __shfl_xor_sync(0xffffffffu, fys, o);
        fzs += __shfl_xor_sync(0xffffffffu, fzs, o);
        phs += __shfl_xor_sync(0xffffffffu, phs, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        h += __shfl_xor_sync(0xffffffffu, h, o);
    }
    const int si = cidx[islot];
    if (g == 0 && si >= 0) {
        if (COUNT) {
            const int ci = perm[si];
            count[ci] = cnt;
            hash[ci] = h;
        } else {
            out[si] = make_float4(pi.w * fxs, pi.w * fys, pi.w * fzs, phs);
        }
    }
    if (VIR) {
        // 1/2 q_i sum_j gsc d (x) d, summed over the warp (fixed tree).  Padding rows contribute
        // nothing: two padding rows of different cells may coincide, so their sums are not used.
        const f2 vv[6] = {vxx, vyy, vzz, vxy, vxz, vyz};
        double v[6];
        #pragma unroll
        for (int c6 = 0; c6 < 6; ++c6) {
            float u0, u1;
            upk(vv[c6], u0, u1);
            v[c6] = si >= 0 ? 0.5 * (double)pi.w * (double)(u0 + u1) : 0.0;
        }
        #pragma unroll
        for (int c6 = 0; c6 < 6; ++c6)
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[c6] += __shfl_xor_sync(0xffffffffu, v[c6], o);
        if (lane == 0)
            for (int c6 = 0; c6 < 6; ++c6) vir[6 * ic + c6] = v[c6];
    }
}

template <int DEG, int NEXP, bool COUNT>
static void launch_cl(int max_clusters, const float4* cpos, const int* cidx, const int* ccell, const float4* bblo,
                      const float4* bbhi, const int* pstart, const int* perm, const NearArgs& a, float4* out,
                      int* count, unsigned long long* hash, cudaStream_t st, double* vir = nullptr)
{
    const int blocks = (max_clusters + 3) / 4;
    if (vir)
        k_near_cl<DEG, NEXP, COUNT, true><<<blocks, 128, 0, st>>>(cpos, cidx, ccell, bblo, bbhi, pstart, perm, a, out,
                                                                   count, hash, vir);
    else
        k_near_cl<DEG, NEXP, COUNT, false><<<blocks, 128, 0, st>>>(cpos, cidx, ccell, bblo, bbhi, pstart, perm, a,
                                                                    out, count, hash, nullptr);
}

/* One explicit Gaussian (the common case: the narrow j = 0 term) unrolled, any other count in a loop. */
template <int DEG>
static void launch_deg(int max_clusters, const float4* cpos, const int* cidx, const int* ccell, const float4* bblo,
                       const float4* bbhi, const int* pstart, const NearArgs& a, float4* out, cudaStream_t st,
                       double* vir)
{
    if (a.n_explicit == 1)
        launch_cl<DEG, 1, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr,
                                 nullptr, st, vir);
    else
        launch_cl<DEG, -1, false>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, nullptr, a, out, nullptr,
                                  nullptr, st, vir);
}

int near_warps(int max_clusters) { return 4 * ((max_clusters + 3) / 4); }

void launch_near(int max_clusters, int deg, const float4* cpos, const int* cidx, const int* ccell, const float4* bblo,
                 const float4* bbhi, const int* pstart, const NearArgs& a, float4* out, cudaStream_t st, double* vir)
{
    switch (deg) {
        case 6: launch_deg<6>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
        case 7: launch_deg<7>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
        case 8: launch_deg<8>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
        case 10: launch_deg<10>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
        case 12: launch_deg<12>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
        case 16: launch_deg<16>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
        case 20: launch_deg<20>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
        default: launch_deg<24>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, a, out, st, vir); break;
    }
}

void launch_pairs(int max_clusters, const float4* cpos, const int* cidx, const int* ccell, const float4* bblo,
                  const float4* bbhi, const int* pstart, const int* perm, const NearArgs& a, int* count,
                  unsigned long long* hash, cudaStream_t st)
{
    launch_cl<8, 0, true>(max_clusters, cpos, cidx, ccell, bblo, bbhi, pstart, perm, a, nullptr, count, hash, st);
}

}  // namespace usr
