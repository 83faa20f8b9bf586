/*
 * k_near.cu -- near part of the u-series, Eq. 20:
 *   N(r) = 1/r - F(r) for r < r_c, 0 otherwise
 *   phi_i^near = sum_j q_j N(r_ij),   F_i^near = q_i sum_j q_j (1/r^3 + F'(r)/r) (r_i - r_j)
 * over all j != i and periodic images.
 *
 * Half-list cluster-pair kernel (k_near_half).  Each cell's atoms come in
 * 8-atom spatial clusters (k_cluster_build), and the clusters of a cell in groups
 * of GI consecutive clusters.  One warp owns one group and walks the j-clusters
 * of its own cell (from the group's first cluster on) and of the 13 neighbour
 * cells whose offset (dz, dy, dx) is lexicographically positive, so that every
 * unordered pair and periodic image is visited exactly once (cells have edge
 * >= r_c and there are >= 3 per axis, so the 27 offsets are distinct images).
 * For 32 candidate j-clusters at a time, each lane tests one candidate's
 * bounding box against the GI i-cluster boxes (a conservative test with the
 * pair distance's rounding); a surviving j-cluster is then evaluated against
 * every i-cluster of the group it reaches, one 8 x 8 step each.
 *
 * Lane layout of a step: lane = (jl = lane % 8, gi = lane / 8) holds j atom jl
 * and the i atoms gi and gi + 4 as a two-wide FP32 pair (add/sub/mul/fma.f32x2),
 * so a step covers all 64 pairs of a cluster pair.  i-side sums stay in
 * registers for the whole walk; j-side sums stay in registers while one
 * j-cluster meets the group's i-clusters, are then reduce-scattered over the
 * four lanes of each j atom (lane gi ends with component gi), and added to the
 * atom's accumulator.  Accumulators are 64-bit integers in fixed point (2^-32):
 * integer addition is associative, so the result is the same bits whatever the
 * order in which warps add their parts (deterministic, no floating-point
 * atomics), and the sum is exact.  Each part is an FP32 sum formed in a fixed
 * order, rounded once to the fixed-point grid.
 *
 * Per pair: r^2 by the single-precision predicate on d = x_i - (x_j + shift);
 * 1/r by rsqrt; F(u = r^2) = explicit narrow Gaussians plus a polynomial in
 * s = 2u / r_c^2 - 1 (Horner, value and derivative).
 *
 * k_pairs_count is the full-list form used only to list pairs: every directed
 * pair (i, j) with the predicate evaluated from i's side, partner counts and
 * index hashes per atom (the canonical list the oracle reproduces bit for bit).
 */
#include <algorithm>

#include "usr_internal.h"

#ifndef USR_NEAR_GI
#define USR_NEAR_GI 4
#endif
#ifndef USR_NEAR_MINB
#define USR_NEAR_MINB 5     // CTAs of 128 threads per SM the register budget is set for (96 registers:
                            // 20 warps per SM, 122 us at r_c = 10 A on the slab against 133 us with 16)
#endif
#ifndef USR_NEAR_NEWTON
#define USR_NEAR_NEWTON 0
#endif

namespace usr {

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Two-wide FP32 arithmetic (the add/mul/fma .f32x2 instructions through
 * CUDA's float2 builtins): each lane evaluates its two pairs of a cluster
 * pair in one instruction stream, halving the issued instructions of the
 * pair arithmetic.  Each element is rounded exactly as the scalar instruction
 * would round it (a - b is formed as a + (-b), which is the same number).
 */
typedef float2 f2;

__device__ __forceinline__ f2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

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

/* ------------------------------------------------------------ half list */

constexpr float kFixScale = 4294967296.0f;   // 2^32 fixed-point units per unit of force or potential
constexpr float kFixMax = 1073741824.0f;     // 2^30: largest magnitude one part may carry

/* Add v to a fixed-point accumulator (nothing for 0; status bit 8 for a part out of range or NaN). */
__device__ __forceinline__ void red_fix(unsigned long long* p, float v, int* status)
{
    if (!(fabsf(v) < kFixMax)) {
        atomicOr(status, 8);
        return;
    }
    const long long q = __float2ll_rn(v * kFixScale);
    if (q != 0) atomicAdd(p, (unsigned long long)q);   // two's complement: a signed add
}

/* One i-cluster of the group, seen by a lane: atoms gi and gi + 4 and their sums. */
struct NearI {
    f2 x, y, z, q;
    f2 fx, fy, fz, ph;
};

struct NearVir {
    f2 xx, yy, zz, xy, xz, yz;
};

/*
 * One 8 x 8 step between i-cluster I and the lane's j atom (xj/yj/zj: minus its
 * position shifted to the image, duplicated into both halves).  Padding rows
 * never pass the distance test: as j atoms they sit near -1e6 (cpos), as i atoms
 * near +1e7 (replaced when the group is loaded).  TRI: the j-cluster is I
 * itself, only pairs with j after i count (tri_a / tri_b for halves a / b).
 */
template <int DEG, int NEXP, bool VIR, bool TRI>
__device__ __forceinline__ void pair_step(const NearArgs& a, NearI& I, f2 xj, f2 yj, f2 zj, float qj, bool tri_a,
                                          bool tri_b, f2& fjx, f2& fjy, f2& fjz, f2& fjp, NearVir& V)
{
    const f2 dx = add2(I.x, xj), dy = add2(I.y, yj), dz = add2(I.z, zj);
    const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    const float r2a = r2.x, r2b = r2.y;
    bool ina = r2a < a.rc2, inb = r2b < a.rc2;
    if (TRI) {
        ina = ina && tri_a;
        inb = inb && tri_b;
    }
    if (!__any_sync(0xffffffffu, ina || inb)) return;
    // pairs outside r_c (or not counted) get r^2 = r_c^2 and charge 0 on both sides: finite, adds 0
    const float ua = ina ? r2a : a.rc2, ub = inb ? r2b : a.rc2;
    const f2 u = pk(ua, ub);
    f2 ri = pk(rsqrt_ftz(ua), rsqrt_ftz(ub));
    if (USR_NEAR_NEWTON) ri = mul2(ri, fma2(mul2(mul2(u, ri), ri), dup(-0.5f), dup(1.5f)));
    // pn = -F(u) and its derivative chain, so that N = 1/r + pn needs no sign change
    const f2 s = fma2(u, dup(a.two_over_rc2), dup(-1.0f));
    f2 pn = dup(a.npoly[DEG]), dpn = pn;
    pn = fma2(pn, s, dup(a.npoly[DEG - 1]));
    #pragma unroll
    for (int d = DEG - 2; d >= 0; --d) {
        dpn = fma2(dpn, s, pn);
        pn = fma2(pn, s, dup(a.npoly[d]));
    }
    f2 d2 = mul2(dpn, dup(a.nd2fac));                                     // 2 dF/du
    const int nexp = NEXP >= 0 ? NEXP : a.n_explicit;
    #pragma unroll
    for (int e = 0; e < nexp; ++e) {
        const f2 t = mul2(u, dup(a.el2[e]));
        const f2 ggn = mul2(pk(exp2_ftz(t.x), exp2_ftz(t.y)), dup(a.nea[e]));   // minus the Gaussian
        pn = add2(pn, ggn);
        d2 = fma2(ggn, dup(a.nne2[e]), d2);
    }
    const f2 nr = add2(ri, pn);                                           // N(r) = 1/r - F
    const f2 g = fma2(mul2(ri, ri), ri, d2);                              // -N'(r) / r
    const float qia = I.q.x, qib = I.q.y;
    const f2 Qj = pk(ina ? qj : 0.f, inb ? qj : 0.f);
    const f2 Qi = pk(ina ? qia : 0.f, inb ? qib : 0.f);
    const f2 gi = mul2(g, Qj);
    I.fx = fma2(gi, dx, I.fx);
    I.fy = fma2(gi, dy, I.fy);
    I.fz = fma2(gi, dz, I.fz);
    I.ph = fma2(nr, Qj, I.ph);
    const f2 gj = mul2(g, Qi);
    fjx = fma2(gj, dx, fjx);
    fjy = fma2(gj, dy, fjy);
    fjz = fma2(gj, dz, fjz);
    fjp = fma2(nr, Qi, fjp);
    if (VIR) {
        // q_i q_j g d (x) d over the pairs (each unordered pair once)
        const f2 w = mul2(gi, I.q);
        const f2 wx = mul2(w, dx), wy = mul2(w, dy);
        V.xx = fma2(wx, dx, V.xx);
        V.xy = fma2(wx, dy, V.xy);
        V.xz = fma2(wx, dz, V.xz);
        V.yy = fma2(wy, dy, V.yy);
        V.yz = fma2(wy, dz, V.yz);
        V.zz = fma2(mul2(w, dz), dz, V.zz);
    }
}

/*
 * The half-shell neighbour cells of a work unit: offsets nb = 13 (the own cell) .. 26 split into
 * kNearSplits ranges of about equal work (the own cell counts half: only j-clusters from the group's
 * first on).
 */
constexpr int kNearSplits = 4;
__constant__ int kSplitLo[kNearSplits] = {13, 17, 20, 23};
__constant__ int kSplitHi[kNearSplits] = {17, 20, 23, 27};

/*
 * One work unit: group `grp` (its GI clusters' i atoms) against the j-clusters of the neighbour
 * offsets nb0 .. nb1 - 1.  Adds the i- and j-side parts to acc; VIR: writes the unit's pair virial
 * sum_pairs d (x) f (six FP64 values) to vir.
 */
template <int GI, int DEG, int NEXP, bool VIR>
__device__ __forceinline__ void near_unit(const ClusterList& L, const NearArgs& a, int grp, int nb0, int nb1,
                                          float4 (*sbox)[2], unsigned long long* __restrict__ acc,
                                          double* __restrict__ vir, int* __restrict__ status)
{
    const int lane = threadIdx.x & 31;
    const int ncx = a.box.nc[0], ncy = a.box.nc[1], ncz = a.box.nc[2];
    if (!USR_IN_BOUNDS(grp, a.max_groups, status)) return;
    const int c0 = L.gfirst[grp];
    if (!USR_IN_BOUNDS(c0, a.max_clusters, status)) return;
    const int cell = L.ccell[c0];
    const int ni = min(GI, (L.pstart[cell + 1] >> 3) - c0);
    if (!USR_IN_BOUNDS(c0 + ni - 1, a.max_clusters, status)) return;
    const int jl = lane & 7, gi = lane >> 3;
    NearI I[GI];
    #pragma unroll
    for (int k = 0; k < GI; ++k) {
        I[k].fx = I[k].fy = I[k].fz = I[k].ph = dup(0.f);
        if (k < ni) {
            // padding rows (index -1) move to +1e7 as i atoms, far from every j position
            const bool va = L.cidx[(c0 + k) * 8 + gi] >= 0, vb = L.cidx[(c0 + k) * 8 + gi + 4] >= 0;
            // group gi of the paired layout: (x, x', y, y') and (z, z', q, q') of atoms gi and gi + 4
            const float4 A = L.cpos[(c0 + k) * 8 + 2 * gi], B = L.cpos[(c0 + k) * 8 + 2 * gi + 1];
            I[k].x = pk(va ? A.x : 1.0e7f, vb ? A.y : 1.0e7f);
            I[k].y = pk(va ? A.z : 1.0e7f, vb ? A.w : 1.0e7f);
            I[k].z = pk(va ? B.x : 1.0e7f, vb ? B.y : 1.0e7f);
            I[k].q = pk(B.z, B.w);
        } else {
            I[k].x = I[k].y = I[k].z = I[k].q = dup(0.f);   // never stepped: its mask bit is never set
        }
    }
    if (lane < 2 * GI) {
        const int k = lane >> 1;
        float4 v;
        if (k < ni) v = (lane & 1) ? L.bbhi[c0 + k] : L.bblo[c0 + k];
        else v = (lane & 1) ? make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f) : make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
        sbox[k][lane & 1] = v;
    }
    __syncwarp();
    NearVir V;
    V.xx = V.yy = V.zz = V.xy = V.xz = V.yz = dup(0.f);
    const bool tri_a = jl > gi, tri_b = jl > gi + 4;
    const int cx = cell % ncx, cy = (cell / ncx) % ncy, cz = cell / (ncx * ncy);
    const float* cf = reinterpret_cast<const float*>(L.cpos);
    // the lane's j atom jl in the paired cluster layout: group jl % 4, half jl / 4
    const int joff = 8 * (jl & 3) + (jl >> 2);
    const bool b1 = (lane & 16) != 0, b0 = (lane & 8) != 0;
    for (int nb = nb0; nb < nb1; ++nb) {
        int nx = cx + nb % 3 - 1, ny = cy + (nb / 3) % 3 - 1, nz = cz + nb / 9 - 1;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        if (nx < 0) { nx += ncx; sx = -a.box.L[0]; } else if (nx >= ncx) { nx -= ncx; sx = a.box.L[0]; }
        if (ny < 0) { ny += ncy; sy = -a.box.L[1]; } else if (ny >= ncy) { ny -= ncy; sy = a.box.L[1]; }
        if (nz < 0) { nz += ncz; sz = -a.box.L[2]; } else if (nz >= ncz) { nz -= ncz; sz = a.box.L[2]; }
        const int nc = (nz * ncy + ny) * ncx + nx;
        const bool own = nb == 13;
        const int jc0 = own ? c0 : L.pstart[nc] >> 3, jc1 = L.pstart[nc + 1] >> 3;
        for (int jb = jc0; jb < jc1; jb += 32) {
            const int jc = jb + lane;
            unsigned int m = 0;
            if (jc < jc1 && USR_IN_BOUNDS(jc, a.max_clusters, status)) {
                const float4 lo = L.bblo[jc], hi = L.bbhi[jc];
                const float lx = __fadd_rn(lo.x, sx), ly = __fadd_rn(lo.y, sy), lz = __fadd_rn(lo.z, sz);
                const float hx = __fadd_rn(hi.x, sx), hy = __fadd_rn(hi.y, sy), hz = __fadd_rn(hi.z, sz);
                #pragma unroll
                for (int k = 0; k < GI; ++k) {
                    const float4 blo = sbox[k][0], bhi = sbox[k][1];
                    // gap between the boxes, rounded like a pair distance
                    const float gx = fmaxf(0.f, fmaxf(__fsub_rn(lx, bhi.x), __fsub_rn(blo.x, hx)));
                    const float gy = fmaxf(0.f, fmaxf(__fsub_rn(ly, bhi.y), __fsub_rn(blo.y, hy)));
                    const float gz = fmaxf(0.f, fmaxf(__fsub_rn(lz, bhi.z), __fsub_rn(blo.z, hz)));
                    if (__fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx))) < a.rc2) m |= 1u << k;
                }
                // own cell: i-cluster c0 + k meets j-clusters from c0 + k on
                if (own && jc - c0 < GI) m &= (2u << (jc - c0)) - 1u;
            }
            unsigned int bal = __ballot_sync(0xffffffffu, m != 0);
            while (bal) {
                const int t = __ffs(bal) - 1;
                bal &= bal - 1;
                const int jcl = jb + t;
                const unsigned int mk = __shfl_sync(0xffffffffu, m, t);
                const float* pj = cf + jcl * 32 + joff;
                // minus the image position, -(x_j + shift): d = x_i + that, the same number as x_i - (x_j + shift)
                const float xj = -__fadd_rn(pj[0], sx), yj = -__fadd_rn(pj[2], sy), zj = -__fadd_rn(pj[4], sz);
                const float qj = pj[6];
                const int sj = L.cidx[jcl * 8 + jl];
                const f2 xj2 = dup(xj), yj2 = dup(yj), zj2 = dup(zj);
                f2 fjx = dup(0.f), fjy = dup(0.f), fjz = dup(0.f), fjp = dup(0.f);
                if (own && jcl - c0 < GI) {
                    // the j-cluster is one of the group's own: that step counts j after i only
                    #pragma unroll
                    for (int k = 0; k < GI; ++k)
                        if (mk & (1u << k)) {
                            if (jcl == c0 + k)
                                pair_step<DEG, NEXP, VIR, true>(a, I[k], xj2, yj2, zj2, qj, tri_a, tri_b, fjx, fjy,
                                                                fjz, fjp, V);
                            else
                                pair_step<DEG, NEXP, VIR, false>(a, I[k], xj2, yj2, zj2, qj, tri_a, tri_b, fjx, fjy,
                                                                 fjz, fjp, V);
                        }
                } else {
                    #pragma unroll
                    for (int k = 0; k < GI; ++k)
                        if (mk & (1u << k))
                            pair_step<DEG, NEXP, VIR, false>(a, I[k], xj2, yj2, zj2, qj, tri_a, tri_b, fjx, fjy, fjz,
                                                             fjp, V);
                }
                // j-side sums: fold the two i halves, reduce-scatter over the four lanes gi of atom jl
                const float vx = fjx.x + fjx.y, vy = fjy.x + fjy.y;
                const float vz = fjz.x + fjz.y, vp = fjp.x + fjp.y;
                const float r0 = __shfl_xor_sync(0xffffffffu, b1 ? vx : vz, 16);
                const float r1 = __shfl_xor_sync(0xffffffffu, b1 ? vy : vp, 16);
                const float k0 = (b1 ? vz : vx) + r0, k1 = (b1 ? vp : vy) + r1;
                const float r2 = __shfl_xor_sync(0xffffffffu, b0 ? k0 : k1, 8);
                const float v = (b0 ? k1 : k0) + r2;                           // component gi of atom jl
                if (sj >= 0 && USR_IN_BOUNDS(sj, a.max_atoms, status))
                    red_fix(acc + 4 * (size_t)sj + gi, gi < 3 ? -qj * v : v, status);
            }
        }
    }
    // i-side sums: reduce-scatter the 8 values of each cluster (2 atoms x 4 components) over the 8
    // lanes jl; lane (jl, gi) ends with component jl % 4 of atom gi + 4 (jl / 4)
    const bool c2 = (lane & 4) != 0, c1 = (lane & 2) != 0, c0b = (lane & 1) != 0;
    #pragma unroll
    for (int k = 0; k < GI; ++k) {
        if (k >= ni) break;
        const float va[4] = {I[k].fx.x, I[k].fy.x, I[k].fz.x, I[k].ph.x};
        const float vb[4] = {I[k].fx.y, I[k].fy.y, I[k].fz.y, I[k].ph.y};
        float w4[4];
        #pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float r = __shfl_xor_sync(0xffffffffu, c2 ? va[m] : vb[m], 4);
            w4[m] = (c2 ? vb[m] : va[m]) + r;
        }
        float w2[2];
        #pragma unroll
        for (int m = 0; m < 2; ++m) {
            const float r = __shfl_xor_sync(0xffffffffu, c1 ? w4[m] : w4[m + 2], 2);
            w2[m] = (c1 ? w4[m + 2] : w4[m]) + r;
        }
        const float r = __shfl_xor_sync(0xffffffffu, c0b ? w2[0] : w2[1], 1);
        const float v = (c0b ? w2[1] : w2[0]) + r;
        const int comp = jl & 3;
        const int slot = (c0 + k) * 8 + gi + 4 * (jl >> 2);
        const int si = L.cidx[slot];
        const float qi = c2 ? I[k].q.y : I[k].q.x;
        if (si >= 0 && USR_IN_BOUNDS(si, a.max_atoms, status))
            red_fix(acc + 4 * (size_t)si + comp, comp < 3 ? qi * v : v, status);
    }
    if (VIR) {
        const f2 vv[6] = {V.xx, V.yy, V.zz, V.xy, V.xz, V.yz};
        double v6[6];
        #pragma unroll
        for (int c6 = 0; c6 < 6; ++c6) v6[c6] = (double)(vv[c6].x + vv[c6].y);
        #pragma unroll
        for (int c6 = 0; c6 < 6; ++c6)
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) v6[c6] += __shfl_xor_sync(0xffffffffu, v6[c6], o);
        if (lane == 0)
            for (int c6 = 0; c6 < 6; ++c6) vir[c6] = v6[c6];
    }
    __syncwarp();   // sbox is rewritten by the warp's next unit
}

/*
 * Persistent warps: each takes work units (group, neighbour range) from a queue counter (zeroed by
 * the cell-list scan), full groups first and the partial ones last, until none is left.  The
 * accumulation is integer, so results do not depend on which warp takes which unit.  acc: 4
 * fixed-point accumulators (Fx, Fy, Fz, phi) per sorted atom, zeroed by k_cluster_build.  VIR: unit u
 * writes its pair virial to vir[6 u ..].
 */
template <int GI, int DEG, int NEXP, bool VIR>
__global__ void __launch_bounds__(128, USR_NEAR_MINB) k_near_half(ClusterList L, NearArgs a, int* __restrict__ queue,
                                                                    unsigned long long* __restrict__ acc,
                                                                    double* __restrict__ vir, int* __restrict__ status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    __shared__ float4 sbox[4][GI][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncell = a.box.nc[0] * a.box.nc[1] * a.box.nc[2];
    const int units = kNearSplits * (L.gfull[ncell] + L.gpart[ncell]);
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(queue, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= units) break;
        const int grp = u / kNearSplits, sub = u - grp * kNearSplits;
        near_unit<GI, DEG, NEXP, VIR>(L, a, grp, kSplitLo[sub], kSplitHi[sub], sbox[warp], acc,
                                      VIR ? vir + 6 * (size_t)u : nullptr, status);
    }
}

/* ------------------------------------------------------------ pair listing */

/*
 * Full list, one warp per i-cluster, lane (il = lane / 4, g = lane % 4) with
 * i atom il and j atoms g and g + 4: partners j != i with r^2 < r_c^2 under the
 * single-precision predicate d = x_i - (x_j + shift), evaluated from i's side;
 * count and the sum of splitmix64 of the partners' caller indices.
 */
__global__ void __launch_bounds__(128) k_pairs_count(ClusterList L, const int* __restrict__ perm, NearArgs a,
                                                     int* __restrict__ count, unsigned long long* __restrict__ hash,
                                                     int* __restrict__ status)
{
    const int ncx = a.box.nc[0], ncy = a.box.nc[1], ncz = a.box.nc[2];
    const int ncl = L.pstart[ncx * ncy * ncz] >> 3;
    const int ic = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ic >= ncl || !USR_IN_BOUNDS(ic, a.max_clusters, status)) return;
    const int il = lane >> 2, g = lane & 3;
    const int islot = ic * 8 + il;
    const float* cf = reinterpret_cast<const float*>(L.cpos);
    const int io = ic * 32 + 8 * (il & 3) + (il >> 2);
    const float4 pi = make_float4(cf[io], cf[io + 2], cf[io + 4], cf[io + 6]);
    const f2 pix = dup(pi.x), piy = dup(pi.y), piz = dup(pi.z);
    const float4 blo = L.bblo[ic], bhi = L.bbhi[ic];
    const int c = L.ccell[ic];
    const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
    int cnt = 0;
    unsigned long long h = 0ull;
    for (int nb = 0; nb < 27; ++nb) {
        int nx = cx + nb % 3 - 1, ny = cy + (nb / 3) % 3 - 1, nz = cz + nb / 9 - 1;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        if (nx < 0) { nx += ncx; sx = -a.box.L[0]; } else if (nx >= ncx) { nx -= ncx; sx = a.box.L[0]; }
        if (ny < 0) { ny += ncy; sy = -a.box.L[1]; } else if (ny >= ncy) { ny -= ncy; sy = a.box.L[1]; }
        if (nz < 0) { nz += ncz; sz = -a.box.L[2]; } else if (nz >= ncz) { nz -= ncz; sz = a.box.L[2]; }
        const f2 sx2 = dup(sx), sy2 = dup(sy), sz2 = dup(sz);
        const int nc = (nz * ncy + ny) * ncx + nx;
        const int jc0 = L.pstart[nc] >> 3, jc1 = L.pstart[nc + 1] >> 3;
        for (int jb = jc0; jb < jc1; jb += 32) {
            const int jc = jb + lane;
            bool near = false;
            if (jc < jc1 && USR_IN_BOUNDS(jc, a.max_clusters, status)) {
                const float4 lo = L.bblo[jc], hi = L.bbhi[jc];
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
                const float4 A = L.cpos[jcl * 8 + 2 * g];     // (x_g, x_g+4, y_g, y_g+4)
                const float4 B = L.cpos[jcl * 8 + 2 * g + 1]; // (z_g, z_g+4, q_g, q_g+4)
                const f2 dx = sub2(pix, add2(pk(A.x, A.y), sx2));
                const f2 dy = sub2(piy, add2(pk(A.z, A.w), sy2));
                const f2 dz = sub2(piz, add2(pk(B.x, B.y), sz2));
                const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                const float r2a = r2.x, r2b = r2.y;
                const bool self = nb == 13 && jcl == ic;
                if (r2a < a.rc2 && !(self && g == il)) {
                    ++cnt;
                    h += mix64((unsigned long long)perm[L.cidx[jcl * 8 + g]]);
                }
                if (r2b < a.rc2 && !(self && g + 4 == il)) {
                    ++cnt;
                    h += mix64((unsigned long long)perm[L.cidx[jcl * 8 + 4 + g]]);
                }
            }
        }
    }
    #pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        h += __shfl_xor_sync(0xffffffffu, h, o);
    }
    const int si = L.cidx[islot];
    if (g == 0 && si >= 0) {
        const int ci = perm[si];
        if (USR_IN_BOUNDS(ci, a.max_atoms, status)) {
            count[ci] = cnt;
            hash[ci] = h;
        }
    }
}

/* ------------------------------------------------------------ launchers */

constexpr int kNearGroup = USR_NEAR_GI;
#ifndef USR_NEAR_RESERVE
#define USR_NEAR_RESERVE 0
#endif

int near_max_groups(int n, int ncell) { return (int)(((long long)n + (8LL * kNearGroup - 1) * ncell) / (8 * kNearGroup)) + 1; }

int near_group_clusters() { return kNearGroup; }

int near_units(int max_groups) { return kNearSplits * max_groups; }

int near_splits() { return kNearSplits; }

/*
 * CTAs per SM the pair kernel's instance can hold, and the SM count (once per instance; thread-safe
 * static initialisation).
 */
template <typename K>
static int2 persistent_shape(K kernel)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0);
    return make_int2(per_sm > 0 ? per_sm : 1, sms > 0 ? sms : 1);
}

/*
 * Grid of the persistent pair kernel: the CTAs the SMs hold at once, less USR_NEAR_RESERVE per SM
 * (slots left for the far-part kernels of the second stream), or at most ctas_per_sm per SM when that
 * is given (the serving loop runs several systems at once); at least one per SM.  Measured on the
 * membrane slab, the pair kernel with every slot (reserve 0) gives the shortest evaluation: it runs
 * 13% faster than with one slot per SM left free, and the far chain, latency-bound, gains less from
 * running beside it than the pair kernel loses.
 */
static int persistent_grid(int2 shape, int ctas_per_sm, int units_max)
{
    int per_sm = shape.x - USR_NEAR_RESERVE;
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    if (per_sm < 1) per_sm = 1;
    return std::max(1, std::min(per_sm * shape.y, (units_max + 3) / 4));
}

template <int GI, int DEG, int NEXP>
static void launch_half(int max_groups, const ClusterList& L, const NearArgs& a, int* queue, unsigned long long* acc,
                        double* vir, int* status, int ctas_per_sm, cudaStream_t st)
{
    const int units_max = kNearSplits * max_groups;
    if (vir) {
        static const int2 shape = persistent_shape(k_near_half<GI, DEG, NEXP, true>);
        launch_pdl(k_near_half<GI, DEG, NEXP, true>, persistent_grid(shape, ctas_per_sm, units_max), 128, 0, st, L,
                   a, queue, acc, vir, status);
    } else {
        static const int2 shape = persistent_shape(k_near_half<GI, DEG, NEXP, false>);
        launch_pdl(k_near_half<GI, DEG, NEXP, false>, persistent_grid(shape, ctas_per_sm, units_max), 128, 0, st, L,
                   a, queue, acc, nullptr, status);
    }
}

/* One explicit Gaussian (the common case: the narrow j = 0 term) unrolled, any other count in a loop. */
template <int DEG>
static void launch_deg(int max_groups, const ClusterList& L, const NearArgs& a, int* queue, unsigned long long* acc,
                       double* vir, int* status, int ctas_per_sm, cudaStream_t st)
{
    if (a.n_explicit == 1)
        launch_half<kNearGroup, DEG, 1>(max_groups, L, a, queue, acc, vir, status, ctas_per_sm, st);
    else
        launch_half<kNearGroup, DEG, -1>(max_groups, L, a, queue, acc, vir, status, ctas_per_sm, st);
}

void launch_near(int max_groups, int deg, const ClusterList& L, const NearArgs& a, int* queue,
                 unsigned long long* acc, double* vir, int* status, int ctas_per_sm, cudaStream_t st)
{
#define USR_NEAR_DEG(D) \
    case D: launch_deg<D>(max_groups, L, a, queue, acc, vir, status, ctas_per_sm, st); break;
    switch (deg) {
        USR_NEAR_DEG(5)
        USR_NEAR_DEG(6)
        USR_NEAR_DEG(7)
        USR_NEAR_DEG(8)
        USR_NEAR_DEG(10)
        USR_NEAR_DEG(12)
        USR_NEAR_DEG(16)
        USR_NEAR_DEG(20)
        default: launch_deg<24>(max_groups, L, a, queue, acc, vir, status, ctas_per_sm, st); break;
    }
#undef USR_NEAR_DEG
}

void launch_pairs(int max_clusters, const ClusterList& L, const int* perm, const NearArgs& a, int* count,
                  unsigned long long* hash, int* status, cudaStream_t st)
{
    const int blocks = (max_clusters + 3) / 4;
    k_pairs_count<<<blocks, 128, 0, st>>>(L, perm, a, count, hash, status);
}

}  // namespace usr
