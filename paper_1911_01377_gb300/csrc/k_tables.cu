/*
 * k_tables.cu -- the convolution tables of a plan, built on the device from
 * the periodised 1D kernels (Eq. 32 deconvolved per term and axis, Eq. 31):
 * every table entry is one value of a term's zero-mean kernel K~ at a
 * circular offset (m - k) mod n, times the term scale on the z axis, so the
 * host uploads only the kernels (N x n values per axis) and the tables are
 * written in parallel.  Values are formed in FP64 and rounded once, exactly
 * as a host-side build would round them.
 *
 *   FP32 path   Bx[k][j nx + m], Ay[j][m][k], Az[m][j nz + k] and the mean rows
 *   tensor-core B tables [batch][tile][NT][K] as hi/lo pairs (TF32 or BF16),
 *               row cols of each tile the DC row (ones, or s_j mu_j on the z pass)
 */
#include <cuda_bf16.h>

#include "usr_internal.h"

namespace usr {

namespace {

__device__ __forceinline__ double kt(const ConvTableArgs& t, int axis, int j, int d)
{
    return t.ktil[((size_t)axis * t.N + j) * t.nmax + d];
}

__device__ __forceinline__ int cmod(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ float tf32_rna(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

}  // namespace

__global__ void __launch_bounds__(256) k_fp32_tables(ConvTableArgs t, float* __restrict__ Bx,
                                                     float* __restrict__ Ay, float* __restrict__ Az,
                                                     float* __restrict__ wx, float* __restrict__ wy,
                                                     float* __restrict__ wz)
{
    const int N = t.N, nx = t.n[0], ny = t.n[1], nz = t.n[2];
    const long long sx = (long long)nx * N * nx, sy = (long long)N * ny * ny, sz = (long long)nz * N * nz;
    const long long total = sx + sy + sz + (long long)N * (nx + ny + nz);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long r = i;
        if (r < sx) {                       // Bx[k][j nx + m]
            const int k = (int)(r / ((long long)N * nx));
            const int jm = (int)(r % ((long long)N * nx));
            const int j = jm / nx, m = jm % nx;
            Bx[r] = (float)kt(t, 0, j, cmod(m - k, nx));
            continue;
        }
        r -= sx;
        if (r < sy) {                       // Ay[j][m][k]
            const int j = (int)(r / ((long long)ny * ny));
            const int mk = (int)(r % ((long long)ny * ny));
            const int m = mk / ny, k = mk % ny;
            Ay[r] = (float)kt(t, 1, j, cmod(m - k, ny));
            continue;
        }
        r -= sy;
        if (r < sz) {                       // Az[m][j nz + k]
            const int m = (int)(r / ((long long)N * nz));
            const int jk = (int)(r % ((long long)N * nz));
            const int j = jk / nz, k = jk % nz;
            Az[r] = (float)(t.scale[j] * kt(t, 2, j, cmod(m - k, nz)));
            continue;
        }
        r -= sz;
        if (r < (long long)N * nx) {
            wx[r] = (float)t.mu[0 * N + r / nx];
            continue;
        }
        r -= (long long)N * nx;
        if (r < (long long)N * ny) {
            wy[r] = (float)t.mu[1 * N + r / ny];
            continue;
        }
        r -= (long long)N * ny;
        const int j = (int)(r / nz);
        wz[r] = (float)(t.scale[j] * t.mu[2 * N + j]);
    }
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_tc_table(ConvTableArgs t, int pass, int batches, int ntiles, int NT,
                                                  int cols, int n_out, int K, void* __restrict__ hi,
                                                  void* __restrict__ lo)
{
    const long long total = (long long)batches * ntiles * NT * K;
    const int N = t.N, nz = t.n[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        const long long row = i / K;
        const int c = (int)(row % NT);
        const int tile = (int)((row / NT) % ntiles);
        const int b = (int)(row / ((long long)NT * ntiles));
        const int m = tile * cols + c;
        double v = 0.0;
        if (c == cols) {                    // DC row
            if (pass == 3) {
                const int j = k / nz;
                v = t.scale[j] * t.mu[2 * N + j];
            } else {
                v = 1.0;
            }
        } else if (c < cols && m < n_out) {
            if (pass == 3) {
                const int j = k / nz, kz = k % nz;
                v = t.scale[j] * kt(t, 2, j, cmod(m - kz, nz));
            } else {
                const int ax = pass - 1, n = t.n[ax];
                v = kt(t, ax, b, cmod(m - k, n));
            }
        }
        if (BF16) {
            const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
            static_cast<__nv_bfloat16*>(hi)[i] = h;
            static_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
        } else {
            const float h = tf32_rna((float)v);
            static_cast<float*>(hi)[i] = h;
            static_cast<float*>(lo)[i] = tf32_rna((float)(v - (double)h));
        }
    }
}

void launch_fp32_tables(const ConvTableArgs& t, float* Bx, float* Ay, float* Az, float* wx, float* wy, float* wz,
                        cudaStream_t st)
{
    k_fp32_tables<<<4 * 152, 256, 0, st>>>(t, Bx, Ay, Az, wx, wy, wz);
}

void launch_tc_table(bool bf16, const ConvTableArgs& t, int pass, int batches, const ConvTcArgs& a, void* hi,
                     void* lo, cudaStream_t st)
{
    if (bf16)
        k_tc_table<true><<<4 * 152, 256, 0, st>>>(t, pass, batches, a.ntiles, a.NT, a.cols, a.n_out, a.K, hi, lo);
    else
        k_tc_table<false><<<4 * 152, 256, 0, st>>>(t, pass, batches, a.ntiles, a.NT, a.cols, a.n_out, a.K, hi, lo);
}

}  // namespace usr
