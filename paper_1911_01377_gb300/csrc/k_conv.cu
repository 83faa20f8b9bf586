/*
 * k_conv.cu -- the separable real-space far-part convolutions (Sec. V,
 * Eqs. 31-32): for each Gaussian term j < N the on-grid potential is the
 * composition of three 1D circular convolutions, and the N results are
 * summed.  Each 1D pass contracts one grid axis with an n x n circulant
 * matrix, so each pass is a (batched) GEMM:
 *
 *   x pass  X_j[z][y][:] = rho[z][y][:] . K_j^x       all terms in one GEMM,
 *           M = ny nz lines, N = N_terms nx, K = nx (the terms share the rho read)
 *   y pass  Y_j[z] = K_j^y . X_j[z]                  batched over (j, z)
 *   z pass  psi = sum_j scale_j K_j^z . Y_j           one GEMM, K = N_terms nz,
 *           the sum over terms is part of the contraction
 *
 * Every 1D kernel is stored as its zero-mean part K~ (circulant) plus its
 * mean mu: K v = K~ v + mu (sum v).  Wide Gaussians are almost constant on
 * the period, so rounding K itself to FP32 would bury their small non-constant
 * part; the split keeps it at full FP32 relative accuracy.  The DC term is the
 * GEMM's rank-one epilogue: row sums of A (x pass, which also subtracts the
 * grid mean: the dropped k = 0 mode) or weighted column sums of B (y, z).
 *
 * This is the plain FP32 CUDA-core form: 64 x 64 x 16 smem tiles, 256
 * threads, 4 x 4 register micro-tiles.
 */
#include "usr_internal.h"

namespace usr {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;
}

template <int MODE>
__global__ void __launch_bounds__(256) k_conv_gemm(ConvGemm g)
{
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    __shared__ float dc[64];
    const int batch = blockIdx.z;
    const int b1 = batch / g.nb2, b2 = batch - b1 * g.nb2;
    const float* __restrict__ A = g.A + b1 * g.a_s1 + b2 * g.a_s2;
    const float* __restrict__ B = g.B + b1 * g.b_s1 + b2 * g.b_s2;
    const float* __restrict__ w = g.dcw ? g.dcw + b1 * g.dcw_s1 : nullptr;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int M = g.M, N = g.N, K = g.K;
    float acc[4][4];
    #pragma unroll
    for (int i = 0; i < 4; ++i)
        #pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    float dcacc = 0.f;
    for (int k0 = 0; k0 < K; k0 += BK) {
        {
            const int r = tid >> 2, kk = (tid & 3) * 4;
            const int m = m0 + r;
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k0 + kk + q;
                As[kk + q][r] = (m < M && k < K) ? __ldg(&A[(long long)m * g.lda + k]) : 0.f;
            }
        }
        {
            const int kr = tid >> 4, c = (tid & 15) * 4;
            const int k = k0 + kr;
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int n = n0 + c + q;
                Bs[kr][c + q] = (k < K && n < N) ? __ldg(&B[(long long)k * g.ldb + n]) : 0.f;
            }
        }
        __syncthreads();
        if (MODE == 1 && tid < BM) {
            #pragma unroll
            for (int kk = 0; kk < BK; ++kk) dcacc += As[kk][tid];
        }
        if (MODE == 2 && tid < BN) {
            #pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const int k = k0 + kk;
                if (k < K) dcacc = fmaf(__ldg(&w[k]), Bs[kk][tid], dcacc);
            }
        }
        #pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
            #pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
            #pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
            #pragma unroll
            for (int i = 0; i < 4; ++i)
                #pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    if (MODE != 0) {
        if (tid < 64) {
            float v = dcacc;
            if (MODE == 1 && g.mean) v -= (float)((double)K * *g.mean);
            dc[tid] = v;
        }
        __syncthreads();
    }
    float* __restrict__ C = g.C + b1 * g.c_s1 + b2 * g.c_s2;
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
        #pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (MODE == 1) v = fmaf(__ldg(&w[n]), dc[ty + 16 * i], v);
            if (MODE == 2) v += dc[tx + 16 * j];
            const int jb = n / g.nsplit;
            const int nn = n - jb * g.nsplit;
            C[jb * g.c_split + (long long)m * g.ldc + nn] = v;
        }
    }
}

void launch_conv(const ConvGemm& g, int batches, cudaStream_t st)
{
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batches);
    switch (g.mode) {
        case 1: k_conv_gemm<1><<<grid, 256, 0, st>>>(g); break;
        case 2: k_conv_gemm<2><<<grid, 256, 0, st>>>(g); break;
        default: k_conv_gemm<0><<<grid, 256, 0, st>>>(g); break;
    }
}

}  // namespace usr
