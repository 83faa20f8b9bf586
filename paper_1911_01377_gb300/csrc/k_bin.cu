/*
 * k_bin.cu -- cell list of the near part (Eq. 20 is range-limited to r_c, so
 * partners of an atom lie in its own or the 26 adjacent cells of edge >= r_c).
 *
 *   bin_count   wrap each position into the box, compute its cell with the
 *               single-precision predicate below, count atoms per cell
 *   scan        exclusive prefix sum of the counts -> cell_start
 *   place       scatter caller indices into their cell's range
 *   cell_sort   order each cell's atoms by caller index (a stable, run-to-run
 *               deterministic order) and gather the sorted float4 rows
 *   clusters    the pair kernel's 8-atom clusters, built from the sorted list
 *
 * Predicate (per axis, RN rounding, no contraction):
 *   k = floorf(x * invL); xw = fmaf(-k, L, x); if (xw < 0) xw += L;
 *   if (xw >= L) xw -= L; cell = min((int)(xw * cs), nc - 1)
 * Non-finite rows, and rows so far from the box (beyond about 2^22 box
 * lengths) that the wrap leaves them outside [0, L], go to cell 0 at the
 * origin with charge 0 and raise the status word.
 */
#include "usr_internal.h"

namespace usr {

__device__ __forceinline__ float canon_wrap(float x, float invL, float L)
{
    float k = floorf(__fmul_rn(x, invL));
    float xw = __fmaf_rn(-k, L, x);
    if (xw < 0.0f) xw = __fadd_rn(xw, L);
    if (xw >= L) xw = __fsub_rn(xw, L);
    return xw;
}

__device__ __forceinline__ int canon_cell(float xw, float cs, int nc)
{
    float u = __fmul_rn(xw, cs);
    int c = (u >= 0.0f) ? (int)u : 0;
    return c > nc - 1 ? nc - 1 : c;
}

__global__ void __launch_bounds__(256) k_bin_count(int n, const float4* __restrict__ xyzq, BoxF b,
                                                   int* __restrict__ count, int* __restrict__ cell_of,
                                                   int* __restrict__ slot, float4* __restrict__ wpos,
                                                   int* __restrict__ status)
{
    pdl_trigger();   // dependents may be scheduled now; they wait for this grid in pdl_wait
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = xyzq[i];
    bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
    float xw = 0.f, yw = 0.f, zw = 0.f;
    if (ok) {
        xw = canon_wrap(p.x, b.invL[0], b.L[0]);
        yw = canon_wrap(p.y, b.invL[1], b.L[1]);
        zw = canon_wrap(p.z, b.invL[2], b.L[2]);
        // Within 2^22 box lengths of the box the period count floorf(x / L) is off by at most one and the
        // wrapped value lies in [0, L] (L itself only by rounding).  Farther out it can be off by more, and
        // a wrapped value outside the box would send the grid kernels' stencils outside their tiles and
        // grids: such rows are refused like non-finite ones (a zero charge at the origin, status bit 1).
        ok = xw >= 0.0f && xw <= b.L[0] && yw >= 0.0f && yw <= b.L[1] && zw >= 0.0f && zw <= b.L[2];
        if (!ok) xw = yw = zw = 0.0f;
    }
    if (!ok || !isfinite(p.w)) atomicOr(status, 1);
    int cx = canon_cell(xw, b.cs[0], b.nc[0]);
    int cy = canon_cell(yw, b.cs[1], b.nc[1]);
    int cz = canon_cell(zw, b.cs[2], b.nc[2]);
    int c = (cz * b.nc[1] + cy) * b.nc[0] + cx;
    if (!USR_IN_BOUNDS(c, b.nc[0] * b.nc[1] * b.nc[2], status)) c = 0;
    cell_of[i] = c;
    // one atomic per distinct cell in the warp (neighbouring caller indices are often in one cell); the slot
    // order inside a cell is arbitrary either way, and k_cell_sort orders each cell by caller index
    const unsigned int peers = __match_any_sync(__activemask(), c);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&count[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    slot[i] = base + __popc(peers & ((1u << lane) - 1u));
    wpos[i] = make_float4(xw, yw, zw, (ok && isfinite(p.w)) ? p.w : 0.0f);
}

/*
 * Exclusive scans, one block of 1024 threads: of count[0..ncell) into
 * start[0..ncell] and of the counts rounded up to a multiple of 8 into
 * pstart[0..ncell] (the padded 8-atom cluster layout of the pair kernels).
 * With gfull given, also the half-list pair kernel's groups of gcl
 * consecutive clusters of one cell: the full groups per cell into
 * gfull[0..ncell], the one partial group a cell may end with into
 * gpart[0..ncell]; and the kernel's work-queue counter is set to zero.
 */
__global__ void __launch_bounds__(1024) k_scan(int ncell, int* __restrict__ count, int* __restrict__ start,
                                               int* __restrict__ pstart, int* __restrict__ gfull,
                                               int* __restrict__ gpart, int gcl, int* __restrict__ queue)
{
    pdl_trigger();   // dependents may be scheduled now; they wait for this grid in pdl_wait
    pdl_wait();
    __shared__ int4 warp_sums[32];
    __shared__ int4 carry;
    if (threadIdx.x == 0) {
        carry = make_int4(0, 0, 0, 0);
        if (queue) *queue = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < ncell ? count[i] : 0;
        if (i < ncell) count[i] = 0;   // ready for the next evaluation's counting
        const int vp = (v + 7) & ~7;
        const int vf = (vp >> 3) / gcl, vq = (vp >> 3) % gcl != 0 ? 1 : 0;
        int4 x = make_int4(v, vp, vf, vq);
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int4 y = make_int4(__shfl_up_sync(0xffffffffu, x.x, o), __shfl_up_sync(0xffffffffu, x.y, o),
                                     __shfl_up_sync(0xffffffffu, x.z, o), __shfl_up_sync(0xffffffffu, x.w, o));
            if (lane >= o) { x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w; }
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int4 w = warp_sums[lane];
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int4 y = make_int4(__shfl_up_sync(0xffffffffu, w.x, o), __shfl_up_sync(0xffffffffu, w.y, o),
                                         __shfl_up_sync(0xffffffffu, w.z, o), __shfl_up_sync(0xffffffffu, w.w, o));
                if (lane >= o) { w.x += y.x; w.y += y.y; w.z += y.z; w.w += y.w; }
            }
            warp_sums[lane] = w;   // inclusive
        }
        __syncthreads();
        const int4 pre = wid > 0 ? warp_sums[wid - 1] : make_int4(0, 0, 0, 0);
        const int4 incl = make_int4(x.x + pre.x + carry.x, x.y + pre.y + carry.y, x.z + pre.z + carry.z,
                                    x.w + pre.w + carry.w);
        if (i < ncell) {
            start[i] = incl.x - v;
            pstart[i] = incl.y - vp;
            if (gfull) {
                gfull[i] = incl.z - vf;
                gpart[i] = incl.w - vq;
            }
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        start[ncell] = carry.x;
        pstart[ncell] = carry.y;
        if (gfull) {
            gfull[ncell] = carry.z;
            gpart[ncell] = carry.w;
        }
    }
}

__global__ void __launch_bounds__(256) k_place(int n, const int* __restrict__ cell_of, const int* __restrict__ slot,
                                               const int* __restrict__ start, int* __restrict__ unsorted,
                                               int* __restrict__ status)
{
    pdl_trigger();   // dependents may be scheduled now; they wait for this grid in pdl_wait
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int d = start[cell_of[i]] + slot[i];
    if (USR_IN_BOUNDS(d, n, status)) unsorted[d] = i;
}

/*
 * One CTA per cell: rank of each entry = number of smaller caller indices in
 * the cell, counted over a shared-memory copy of the cell's entries (all
 * threads read the same element at a time: broadcast, no bank conflicts).
 * Cells larger than the shared copy fall back to counting in global memory.
 */
constexpr int kSortThreads = 128;
constexpr int kSortMax = 2048;

__global__ void __launch_bounds__(kSortThreads) k_cell_sort(int n, const int* __restrict__ start,
                                                            const int* __restrict__ unsorted,
                                                            const float4* __restrict__ wpos, int* __restrict__ perm,
                                                            float4* __restrict__ spos, int* __restrict__ status)
{
    pdl_trigger();   // dependents may be scheduled now; they wait for this grid in pdl_wait
    pdl_wait();
    __shared__ int v[kSortMax];
    const int c = blockIdx.x;
    const int s0 = start[c], m = start[c + 1] - s0;
    if (m == 0) return;
    const bool in_smem = m <= kSortMax;
    if (in_smem)
        for (int e = threadIdx.x; e < m; e += kSortThreads) v[e] = unsorted[s0 + e];
    __syncthreads();
    const int* src = in_smem ? v : unsorted + s0;
    for (int e = threadIdx.x; e < m; e += kSortThreads) {
        const int x = src[e];
        int r = 0;
        for (int f = 0; f < m; ++f) r += src[f] < x;
        if (!USR_IN_BOUNDS(s0 + r, n, status) || !USR_IN_BOUNDS(x, n, status)) continue;
        perm[s0 + r] = x;
        spos[s0 + r] = wpos[x];
    }
}

/*
 * 8-atom clusters for the pair kernel, one CTA per cell: the cell's atoms
 * are ordered by the Morton code of their position on an 8 x 8 x 8 lattice
 * inside the cell (ties by sorted index), so that runs of 8 are compact;
 * written to the padded layout at pstart[c] with dummy rows (q = 0, far
 * away and far apart, index -1) after the last atom; then each cluster's
 * bounding box.
 *
 * Cluster positions are stored paired for the pair kernel's two-wide FP32
 * arithmetic: atom t of a cluster (t = 4 h + g, h = 0, 1) goes to the 32-byte
 * group g as x at float 8 g + h, y at 8 g + 2 + h, z at 8 g + 4 + h and q at
 * 8 g + 6 + h, so one lane's two 16-byte loads give (x_g, x_g+4), (y_g, y_g+4),
 * (z_g, z_g+4), (q_g, q_g+4).
 */
__device__ __forceinline__ int spread3(int v)
{
    return (v & 1) | ((v & 2) << 2) | ((v & 4) << 4);
}

__device__ __forceinline__ int pk_off(int slot)
{
    const int t = slot & 7;
    return (slot >> 3) * 32 + 8 * (t & 3) + (t >> 2);
}

__device__ __forceinline__ void pk_store(float* cp, int slot, float4 p)
{
    const int o = pk_off(slot);
    cp[o] = p.x;
    cp[o + 2] = p.y;
    cp[o + 4] = p.z;
    cp[o + 6] = p.w;
}

__device__ __forceinline__ int morton_key(float4 p, float ox, float oy, float oz, float kx, float ky, float kz)
{
    const int ix = min(7, max(0, (int)((p.x - ox) * kx)));
    const int iy = min(7, max(0, (int)((p.y - oy) * ky)));
    const int iz = min(7, max(0, (int)((p.z - oz) * kz)));
    return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

/*
 * The clusters of one cell per CTA, from the sorted cell list (k_cell_sort):
 * Morton order as above, the padded paired layout, each cluster's bounding
 * box; also the first cluster of each of the cell's groups of gcl clusters,
 * and the cell's rows of the pair kernel's fixed-point accumulators set to
 * zero.  A separate kernel from the sort, so that the far part, which needs
 * only the sorted list, can start beside it on another stream.
 */
__global__ void __launch_bounds__(kSortThreads) k_cluster_build(const int* __restrict__ start,
                                                                const int* __restrict__ pstart,
                                                                const int* __restrict__ gfull,
                                                                const int* __restrict__ gpart, int gcl, BoxF b,
                                                                const float4* __restrict__ spos,
                                                                int* __restrict__ key, float4* __restrict__ cpos,
                                                                int* __restrict__ cidx, int* __restrict__ ccell,
                                                                float4* __restrict__ bblo, float4* __restrict__ bbhi,
                                                                int* __restrict__ gfirst,
                                                                unsigned long long* __restrict__ acc, int n,
                                                                int max_slots, int max_groups,
                                                                int* __restrict__ status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    __shared__ int ks[kSortMax];
    const int c = blockIdx.x;
    const int s0 = start[c], m = start[c + 1] - s0;
    const int p0 = pstart[c], pm = pstart[c + 1] - p0;
    if (pm == 0) return;                                  // an empty cell has no clusters
    const int cx = c % b.nc[0], cy = (c / b.nc[0]) % b.nc[1], cz = c / (b.nc[0] * b.nc[1]);
    const float ox = (float)cx / b.cs[0], oy = (float)cy / b.cs[1], oz = (float)cz / b.cs[2];
    const float kx = 8.0f * b.cs[0], ky = 8.0f * b.cs[1], kz = 8.0f * b.cs[2];
    const bool in_smem = m <= kSortMax;
    float* cp = reinterpret_cast<float*>(cpos);
    {
        // full groups in cell order, then the partial ones (the pair kernel takes them in that order,
        // so its last work units are the small ones)
        const int f0 = gfull[c], nf = gfull[c + 1] - f0;
        for (int k = threadIdx.x; k < nf; k += kSortThreads)
            if (USR_IN_BOUNDS(f0 + k, max_groups, status)) gfirst[f0 + k] = (p0 >> 3) + k * gcl;
        if (threadIdx.x == 0 && gpart[c + 1] > gpart[c]) {
            const int gp = gfull[b.nc[0] * b.nc[1] * b.nc[2]] + gpart[c];
            if (USR_IN_BOUNDS(gp, max_groups, status)) gfirst[gp] = (p0 >> 3) + nf * gcl;
        }
        if (USR_IN_BOUNDS(s0 + m - 1, n, status)) {
            ulonglong2* a2 = reinterpret_cast<ulonglong2*>(acc + 4 * (size_t)s0);
            for (int e = threadIdx.x; e < 2 * m; e += kSortThreads) a2[e] = make_ulonglong2(0ull, 0ull);
        }
    }
    int* kk = in_smem ? ks : key + s0;
    if (!USR_IN_BOUNDS(s0 + m - 1, n, status)) return;
    // cluster order: Morton code of each atom on an 8 x 8 x 8 lattice inside the cell, ties by sorted index
    for (int e = threadIdx.x; e < m; e += kSortThreads) kk[e] = morton_key(spos[s0 + e], ox, oy, oz, kx, ky, kz);
    __syncthreads();
    for (int e = threadIdx.x; e < m; e += kSortThreads) {
        const int ke = kk[e];
        int r = 0;
        for (int f = 0; f < m; ++f) {
            const int kf = kk[f];
            r += (kf < ke) || (kf == ke && f < e);
        }
        if (!USR_IN_BOUNDS(p0 + r, max_slots, status)) continue;
        pk_store(cp, p0 + r, spos[s0 + e]);
        cidx[p0 + r] = s0 + e;
    }
    for (int e = m + threadIdx.x; e < pm; e += kSortThreads) {
        if (!USR_IN_BOUNDS(p0 + e, max_slots, status)) continue;
        // padding rows: far from the box, so never within r_c of an atom, and 4e4 A apart within
        // a cluster (rows of different cells may coincide; the pair kernel never uses their sums)
        const float far = -1.0e6f - 4.0e4f * (float)(e & 7);
        pk_store(cp, p0 + e, make_float4(far, far, far, 0.0f));
        cidx[p0 + e] = -1;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < (pm >> 3); k += kSortThreads) {
        float4 lo = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f), hi = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
        for (int t = 0; t < 8; ++t) {
            const int sl = p0 + 8 * k + t;
            if (cidx[sl] < 0) continue;
            const int o = pk_off(sl);
            const float4 p = make_float4(cp[o], cp[o + 2], cp[o + 4], 0.f);
            lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
            hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
        }
        const int cl = (p0 >> 3) + k;
        if (!USR_IN_BOUNDS(cl, max_slots >> 3, status)) continue;
        bblo[cl] = lo;
        bbhi[cl] = hi;
        ccell[cl] = c;
    }
}

cudaError_t launch_bin(int n, const float4* xyzq, const BoxF& b, int ncell, int* count, int* cell_of, int* slot,
                       float4* wpos, int* cell_start, int* pstart, int* unsorted, int* perm, float4* spos,
                       int* status, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncell, st);
    if (e != cudaSuccess) return e;
    int nb = (n + 255) / 256;
    k_bin_count<<<nb, 256, 0, st>>>(n, xyzq, b, count, cell_of, slot, wpos, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_scan<<<1, 1024, 0, st>>>(ncell, count, cell_start, pstart, nullptr, nullptr, 1, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_place<<<nb, 256, 0, st>>>(n, cell_of, slot, cell_start, unsorted, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_cell_sort<<<ncell, kSortThreads, 0, st>>>(n, cell_start, unsorted, wpos, perm, spos, status);
    return cudaGetLastError();
}

/* The sorted cell list: counts, scan (with the pair kernel's group counts), placement, per-cell sort. */
void launch_bin_sorted(int n, const float4* xyzq, const BoxF& b, int ncell, int* count, int* cell_of, int* slot,
                       float4* wpos, int* cell_start, int* pstart, int* gfull, int* gpart, int* queue, int* unsorted,
                       int* perm, float4* spos, int* status, cudaStream_t st)
{
    // count[] is zero on entry: the context zeroes it when it is (re)configured, and k_scan zeroes every
    // entry after reading it, ready for the next evaluation (no memset between the kernels)
    const int gcl = near_group_clusters();
    int nb = (n + 255) / 256;
    launch_pdl(k_bin_count, nb, 256, 0, st, n, xyzq, b, count, cell_of, slot, wpos, status);
    launch_pdl(k_scan, 1, 1024, 0, st, ncell, count, cell_start, pstart, gfull, gpart, gcl, queue);
    launch_pdl(k_place, nb, 256, 0, st, n, cell_of, slot, cell_start, unsorted, status);
    launch_pdl(k_cell_sort, ncell, kSortThreads, 0, st, n, cell_start, unsorted, wpos, perm, spos, status);
}

/* The pair kernels' clusters from the sorted cell list (slot[] of launch_bin_sorted is reused for keys). */
void launch_clusters(int n, const BoxF& b, int ncell, const int* cell_start, const int* pstart, const int* gfull,
                     const int* gpart, int* gfirst, const float4* spos, int* key, float4* cpos, int* cidx,
                     int* ccell, float4* bblo, float4* bbhi, unsigned long long* near_acc, int max_clusters,
                     int max_groups, int* status, cudaStream_t st)
{
    launch_pdl(k_cluster_build, ncell, kSortThreads, 0, st, cell_start, pstart, gfull, gpart, near_group_clusters(),
               b, spos, key, cpos, cidx, ccell, bblo, bbhi, gfirst, near_acc, n, 8 * max_clusters, max_groups,
               status);
}

}  // namespace usr
