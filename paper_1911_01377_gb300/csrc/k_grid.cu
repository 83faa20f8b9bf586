/*
 * k_grid.cu -- the particle-grid legs of the far part (Sec. V with Gaussian
 * spreading, the GSE scheme named in Sec. IV.A):
 *
 *   spread   rho_g = sum_i q_i exp(-|g - r_i|^2 / (2 sigma_s^2)) on a P^3
 *            stencil around each charge (normalisation is folded into the
 *            convolution scale).  Atomic-free in global memory: each CTA owns
 *            an 8^3 brick of grid points, visits the sorted atoms of the cells
 *            whose stencils can reach the brick and accumulates into shared
 *            memory; one warp per atom, lanes over the stencil's (x, y)
 *            columns.  The last CTA also reduces the grid mean (the k = 0
 *            mode, dropped per Eq. 4).
 *   gather   phi_far,i = sum_g w(g - r_i) psi_g and F_far,i = -q_i grad phi_far,i
 *            (the second spreading Gaussian of Eq. 32's 1/|S(k)|^2), one warp
 *            per atom; adds the near part and the self term -F(0) q_i, writes
 *            (F, phi) in caller order and reduces the energies
 *            E = 1/2 sum q_i phi_i (and its near / far / self parts) in FP64.
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

/* Grid coordinate of a wrapped position: base point g0 = floor(u), fraction t. */
__device__ __forceinline__ void grid_coord(float xw, float gs, int& g0, float& t)
{
    float u = xw * gs;
    float f = floorf(u);
    g0 = (int)f;
    t = u - f;
}

}  // namespace

template <int P>
__global__ void __launch_bounds__(256) k_spread(const float4* __restrict__ pos, const int* __restrict__ cell_start,
                                                GridArgs g, float* __restrict__ rho, double* __restrict__ partial,
                                                unsigned int* __restrict__ counter, double* __restrict__ mean)
{
    constexpr int B = kBrick;
    constexpr int H = P / 2;
    __shared__ float sm[B * B * B];
    __shared__ double red[8];
    __shared__ int is_last;
    const int n0 = g.box.n[0], n1 = g.box.n[1], n2 = g.box.n[2];
    const int nbx = (n0 + B - 1) / B, nby = (n1 + B - 1) / B;
    const int bid = blockIdx.x;
    const int x0 = (bid % nbx) * B, y0 = ((bid / nbx) % nby) * B, z0 = (bid / (nbx * nby)) * B;
    const int ex0 = min(B, n0 - x0), ex1 = min(B, n1 - y0), ex2 = min(B, n2 - z0);
    for (int t = threadIdx.x; t < B * B * B; t += 256) sm[t] = 0.f;
    // cells whose atoms can reach the brick: stencil base g0 in [o - H, o + ext + H - 2]
    int clo[3], ccnt[3];
    const int org[3] = {x0, y0, z0}, ext[3] = {ex0, ex1, ex2};
    #pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = (float)(org[a] - H) / g.box.gs[a] - 1e-3f;
        const float hi = (float)(org[a] + ext[a] + H - 1) / g.box.gs[a] + 1e-3f;
        const int c0 = (int)floorf(lo * g.box.cs[a]);
        const int c1 = (int)floorf(hi * g.box.cs[a]);
        clo[a] = c0;
        ccnt[a] = min(c1 - c0 + 1, g.box.nc[a]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int iz = 0; iz < ccnt[2]; ++iz) {
        int cz = clo[2] + iz;
        cz = ((cz % g.box.nc[2]) + g.box.nc[2]) % g.box.nc[2];
        for (int iy = 0; iy < ccnt[1]; ++iy) {
            int cy = clo[1] + iy;
            cy = ((cy % g.box.nc[1]) + g.box.nc[1]) % g.box.nc[1];
            for (int ix = 0; ix < ccnt[0]; ++ix) {
                int cx = clo[0] + ix;
                cx = ((cx % g.box.nc[0]) + g.box.nc[0]) % g.box.nc[0];
                const int c = (cz * g.box.nc[1] + cy) * g.box.nc[0] + cx;
                const int as = cell_start[c], ae = cell_start[c + 1];
                for (int ai = as + warp; ai < ae; ai += 8) {
                    const float4 p = pos[ai];
                    int d[3];
                    float t[3];
                    const float pc[3] = {p.x, p.y, p.z};
                    bool hit = true;
                    #pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        int g0;
                        grid_coord(pc[a], g.box.gs[a], g0, t[a]);
                        int dd = g0 - org[a];
                        const int nn = g.box.n[a];
                        if (dd < -H) dd += nn;
                        else if (dd > ext[a] + H - 2) dd -= nn;
                        hit = hit && dd >= -H && dd <= ext[a] + H - 2;
                        d[a] = dd;
                    }
                    if (!hit) continue;
                    // stencil index l in [0, P) sits at brick offset d - H + 1 + l
                    int l0[3], l1[3];
                    #pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        l0[a] = max(0, H - 1 - d[a]);
                        l1[a] = min(P, ext[a] + H - 1 - d[a]);
                    }
                    float wx = 0.f, wy = 0.f, wz = 0.f;
                    if (lane < P) {
                        const float o = (float)(lane - H + 1);
                        float dx = o - t[0], dy = o - t[1], dz = o - t[2];
                        wx = p.w * __expf(-dx * dx * g.hh[0]);
                        wy = __expf(-dy * dy * g.hh[1]);
                        wz = __expf(-dz * dz * g.hh[2]);
                    }
                    const int exn = l1[0] - l0[0];
                    const int npair = exn * (l1[1] - l0[1]);
                    const int bxo = d[0] - H + 1, byo = d[1] - H + 1, bzo = d[2] - H + 1;
                    for (int pb = 0; pb < npair; pb += 32) {
                        const int pp = pb + lane;
                        const bool valid = pp < npair;
                        const int q = valid ? pp : 0;
                        const int jy = q / exn;
                        const int jx = q - jy * exn + l0[0];
                        const int ly = jy + l0[1];
                        const float wxy = __shfl_sync(0xffffffffu, wx, jx) * __shfl_sync(0xffffffffu, wy, ly);
                        const int off = (byo + ly) * B + (bxo + jx);
                        #pragma unroll
                        for (int lz = 0; lz < P; ++lz) {
                            const float wzv = __shfl_sync(0xffffffffu, wz, lz);
                            if (valid && lz >= l0[2] && lz < l1[2]) atomicAdd(&sm[(bzo + lz) * B * B + off], wxy * wzv);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    double local = 0.0;
    for (int t = threadIdx.x; t < B * B * B; t += 256) {
        const int x = t % B, y = (t / B) % B, z = t / (B * B);
        if (x < ex0 && y < ex1 && z < ex2) {
            const float v = sm[t];
            rho[((size_t)(z0 + z) * n1 + (y0 + y)) * n0 + (x0 + x)] = v;
            local += v;
        }
    }
    local = warp_sum_d(local);
    if (lane == 0) red[warp] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        partial[bid] = s;
        __threadfence();
        unsigned int ticket = atomicAdd(counter, 1u);
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
__global__ void __launch_bounds__(256) k_gather(int n, const float4* __restrict__ pos, const int* __restrict__ perm,
                                                const float4* __restrict__ near_out, const float* __restrict__ psi,
                                                GridArgs g, float4* __restrict__ out, float4* __restrict__ near_dbg,
                                                float4* __restrict__ far_dbg, double* __restrict__ partial,
                                                unsigned int* __restrict__ counter, double* __restrict__ energy)
{
    constexpr int H = P / 2;
    __shared__ double red[8][4];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x * 8 + warp;
    double e_tot = 0.0, e_near = 0.0, e_far = 0.0, e_self = 0.0;
    if (s < n) {
        const int n0 = g.box.n[0], n1 = g.box.n[1], n2 = g.box.n[2];
        const float4 p = pos[s];
        int gb[3];
        float t[3];
        const float pc[3] = {p.x, p.y, p.z};
        #pragma unroll
        for (int a = 0; a < 3; ++a) {
            int g0;
            grid_coord(pc[a], g.box.gs[a], g0, t[a]);
            gb[a] = g0 - H + 1;
        }
        float wx = 0.f, wy = 0.f, wz = 0.f, dwx = 0.f, dwy = 0.f, dwz = 0.f;
        if (lane < P) {
            const float o = (float)(lane - H + 1);
            const float dx = o - t[0], dy = o - t[1], dz = o - t[2];
            wx = __expf(-dx * dx * g.hh[0]);
            wy = __expf(-dy * dy * g.hh[1]);
            wz = __expf(-dz * dz * g.hh[2]);
            dwx = wx * dx * g.dfac[0];
            dwy = wy * dy * g.dfac[1];
            dwz = wz * dz * g.dfac[2];
        }
        float aphi = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
        for (int pb = 0; pb < P * P; pb += 32) {
            const int pp = pb + lane;
            const bool valid = pp < P * P;
            const int q = valid ? pp : 0;
            const int jy = q / P, jx = q - jy * P;
            const float wxv = __shfl_sync(0xffffffffu, wx, jx);
            const float wyv = __shfl_sync(0xffffffffu, wy, jy);
            const float dwxv = __shfl_sync(0xffffffffu, dwx, jx);
            const float dwyv = __shfl_sync(0xffffffffu, dwy, jy);
            int gx = gb[0] + jx, gy = gb[1] + jy;
            if (gx < 0) gx += n0; else if (gx >= n0) gx -= n0;
            if (gy < 0) gy += n1; else if (gy >= n1) gy -= n1;
            const int row = gy * n0 + gx;
            const float wxy = wxv * wyv, cx = dwxv * wyv, cy = wxv * dwyv;
            #pragma unroll
            for (int lz = 0; lz < P; ++lz) {
                const float wzv = __shfl_sync(0xffffffffu, wz, lz);
                const float dwzv = __shfl_sync(0xffffffffu, dwz, lz);
                int gz = gb[2] + lz;
                if (gz < 0) gz += n2; else if (gz >= n2) gz -= n2;
                if (valid) {
                    const float v = __ldg(&psi[(size_t)gz * n0 * n1 + row]);
                    const float tv = v * wzv;
                    aphi = fmaf(wxy, tv, aphi);
                    ax = fmaf(cx, tv, ax);
                    ay = fmaf(cy, tv, ay);
                    az = fmaf(wxy * dwzv, v, az);
                }
            }
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
            e_near = 0.5 * (double)qi * (double)nr.w;
            e_far = 0.5 * (double)qi * (double)aphi;
            e_self = -0.5 * (double)g.F0 * (double)qi * (double)qi;
            e_tot = e_near + e_far + e_self;
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
        unsigned int ticket = atomicAdd(counter, 1u);
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

int gather_blocks(int n) { return (n + 7) / 8; }

void launch_spread(int P, const float4* spos, const int* cell_start, const GridArgs& g, float* rho, double* partial,
                   unsigned int* counter, double* mean, cudaStream_t st)
{
    const int nb = ((g.box.n[0] + kBrick - 1) / kBrick) * ((g.box.n[1] + kBrick - 1) / kBrick) *
                   ((g.box.n[2] + kBrick - 1) / kBrick);
    switch (P) {
        case 8: k_spread<8><<<nb, 256, 0, st>>>(spos, cell_start, g, rho, partial, counter, mean); break;
        case 10: k_spread<10><<<nb, 256, 0, st>>>(spos, cell_start, g, rho, partial, counter, mean); break;
        case 12: k_spread<12><<<nb, 256, 0, st>>>(spos, cell_start, g, rho, partial, counter, mean); break;
        case 14: k_spread<14><<<nb, 256, 0, st>>>(spos, cell_start, g, rho, partial, counter, mean); break;
        default: k_spread<16><<<nb, 256, 0, st>>>(spos, cell_start, g, rho, partial, counter, mean); break;
    }
}

void launch_gather(int P, int n, const float4* spos, const int* perm, const float4* near_out, const float* psi,
                   const GridArgs& g, float4* out, float4* near_dbg, float4* far_dbg, double* partial,
                   unsigned int* counter, double* energy, cudaStream_t st)
{
    const int nb = gather_blocks(n);
    switch (P) {
        case 8: k_gather<8><<<nb, 256, 0, st>>>(n, spos, perm, near_out, psi, g, out, near_dbg, far_dbg, partial, counter, energy); break;
        case 10: k_gather<10><<<nb, 256, 0, st>>>(n, spos, perm, near_out, psi, g, out, near_dbg, far_dbg, partial, counter, energy); break;
        case 12: k_gather<12><<<nb, 256, 0, st>>>(n, spos, perm, near_out, psi, g, out, near_dbg, far_dbg, partial, counter, energy); break;
        case 14: k_gather<14><<<nb, 256, 0, st>>>(n, spos, perm, near_out, psi, g, out, near_dbg, far_dbg, partial, counter, energy); break;
        default: k_gather<16><<<nb, 256, 0, st>>>(n, spos, perm, near_out, psi, g, out, near_dbg, far_dbg, partial, counter, energy); break;
    }
}

}  // namespace usr
