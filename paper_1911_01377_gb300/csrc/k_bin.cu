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
 *
 * Predicate (per axis, RN rounding, no contraction):
 *   k = floorf(x * invL); xw = fmaf(-k, L, x); if (xw < 0) xw += L;
 *   if (xw >= L) xw -= L; cell = min((int)(xw * cs), nc - 1)
 * Non-finite rows go to cell 0 at the origin and raise the status word.
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
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = xyzq[i];
    bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
    float xw = 0.f, yw = 0.f, zw = 0.f;
    if (ok) {
        xw = canon_wrap(p.x, b.invL[0], b.L[0]);
        yw = canon_wrap(p.y, b.invL[1], b.L[1]);
        zw = canon_wrap(p.z, b.invL[2], b.L[2]);
    }
    if (!ok || !isfinite(p.w)) atomicOr(status, 1);
    int cx = canon_cell(xw, b.cs[0], b.nc[0]);
    int cy = canon_cell(yw, b.cs[1], b.nc[1]);
    int cz = canon_cell(zw, b.cs[2], b.nc[2]);
    int c = (cz * b.nc[1] + cy) * b.nc[0] + cx;
    cell_of[i] = c;
    slot[i] = atomicAdd(&count[c], 1);
    wpos[i] = make_float4(xw, yw, zw, (ok && isfinite(p.w)) ? p.w : 0.0f);
}

/* Exclusive scan of count[0..ncell) into start[0..ncell], one block of 1024 threads. */
__global__ void __launch_bounds__(1024) k_scan(int ncell, const int* __restrict__ count, int* __restrict__ start)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < ncell ? count[i] : 0;
        int x = v;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = warp_sums[lane];
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;   // inclusive
        }
        __syncthreads();
        int incl = x + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
        if (i < ncell) start[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void __launch_bounds__(256) k_place(int n, const int* __restrict__ cell_of, const int* __restrict__ slot,
                                               const int* __restrict__ start, int* __restrict__ unsorted)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsorted[start[cell_of[i]] + slot[i]] = i;
}

/* One warp per cell: rank of each entry = number of smaller caller indices in the cell. */
__global__ void __launch_bounds__(256) k_cell_sort(int ncell, const int* __restrict__ start,
                                                   const int* __restrict__ unsorted, const float4* __restrict__ wpos,
                                                   int* __restrict__ perm, float4* __restrict__ spos)
{
    int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const int lane = threadIdx.x & 31;
    const int s0 = start[c], m = start[c + 1] - s0;
    for (int e = lane; e < m; e += 32) {
        int v = unsorted[s0 + e];
        int r = 0;
        for (int f = 0; f < m; ++f) r += unsorted[s0 + f] < v;
        perm[s0 + r] = v;
        spos[s0 + r] = wpos[v];
    }
}

void launch_bin(int n, const float4* xyzq, const BoxF& b, int ncell, int* count, int* cell_of, int* slot,
                float4* wpos, int* cell_start, int* unsorted, int* perm, float4* spos, int* status,
                cudaStream_t st)
{
    cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncell, st);
    int nb = (n + 255) / 256;
    k_bin_count<<<nb, 256, 0, st>>>(n, xyzq, b, count, cell_of, slot, wpos, status);
    k_scan<<<1, 1024, 0, st>>>(ncell, count, cell_start);
    k_place<<<nb, 256, 0, st>>>(n, cell_of, slot, cell_start, unsorted);
    k_cell_sort<<<(ncell + 7) / 8, 256, 0, st>>>(ncell, cell_start, unsorted, wpos, perm, spos);
}

}  // namespace usr
