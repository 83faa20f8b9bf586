/*
 * k_multilevel.cu -- the grid transfers of the multilevel far part (Sec. V:
 * wider Gaussian terms can be handled on coarser grids).  The wide terms are
 * convolved on a grid of half the points per axis; per axis the fine kernel
 * e_w is the product w / (2 pi a b c) (e_b * e_c * e_a), applied as
 *
 *   restriction   r(G) = sum_g  eR(g - 2G) f(g)        (fine -> coarse, width a)
 *   coarse pass   t(G) = sum_G' e_c((G - G') H) r(G')   (the ordinary 1D passes)
 *   prolongation  f(g) = sum_G  eP(g - 2G) t(G)        (coarse -> fine, width b)
 *
 * with the constant factors in the coarse term scale.  The weights are banded
 * (|g - 2G| <= kMlT, 33 taps, the same for every grid since a = b = 2.6 h) and
 * periodic; they travel in the kernel parameters, so every tap is one FMA
 * with a constant-bank operand.
 *
 * Each CTA (8 warps) stages a window of its input along the transfer axis in
 * shared memory as [row = position along the axis][32 columns], loaded with
 * coalesced rows (for the x axis the 32 columns are 32 lines, transposed on
 * the way in and out).  A lane owns one column and four consecutive outputs,
 * read from a register window of the rows they share: 39 shared loads per
 * four restricted outputs (132 taps), 18 per four prolonged ones.
 */
#include "usr_internal.h"

namespace usr {

namespace {

constexpr int kMlCh = 32;                        // outputs along the axis per CTA (8 warps x 4)
constexpr int kMlWinR = 2 * kMlCh + 2 * kMlT - 1; // restriction: fine rows feeding 32 coarse outputs
constexpr int kMlWinP = kMlCh / 2 + kMlT;         // prolongation: coarse rows feeding 32 fine outputs
constexpr int kMlPad = 33;                        // row stride of the staged window (conflict-free columns)

__device__ __forceinline__ int wrap(int g, int n)
{
    g %= n;
    return g < 0 ? g + n : g;
}

__device__ __forceinline__ float tf32_rna(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

/*
 * Element offsets for a [d2][d1][d0] array whose extent along AX is `na` (the other two are d0..d2 of the
 * output): `col` is x (AX = 1, 2) or the line index y + d1 z (AX = 0), `g` the position along AX.
 */
template <int AX>
__device__ __forceinline__ long long offs(int col, int g, int b, int d0, int d1, int na)
{
    if (AX == 0) return (long long)col * na + g;                          // lines of length na
    if (AX == 1) return ((long long)b * na + g) * d0 + col;               // b = z
    return ((long long)g * d1 + b) * d0 + col;                            // b = y
}

/*
 * Stage rows [g0, g0 + ROWS) (periodic in n_in) of 32 columns starting at col0 into S[row][col].  Columns
 * past ncol read as zero.  All of a thread's loads are issued before its shared-memory stores.
 */
template <int AX, int ROWS>
__device__ __forceinline__ void stage(float (*S)[kMlPad], const float* __restrict__ in, int g0, int n_in,
                                      int col0, int ncol, int b, int d0, int d1)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (AX == 0) {
        // warp w loads lines w, w + 8, w + 16, w + 24; lanes run along the line
        constexpr int PER = (ROWS + 31) / 32;
        float v[4][PER];
        #pragma unroll
        for (int li = 0; li < 4; ++li) {
            const int l = warp + 8 * li;
            const bool ok = col0 + l < ncol;
            #pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int r = lane + 32 * k;
                v[li][k] = ok && r < ROWS ? in[offs<0>(col0 + l, wrap(g0 + r, n_in), b, d0, d1, n_in)] : 0.f;
            }
        }
        #pragma unroll
        for (int li = 0; li < 4; ++li)
            #pragma unroll
            for (int k = 0; k < PER; ++k)
                if (lane + 32 * k < ROWS) S[lane + 32 * k][warp + 8 * li] = v[li][k];
    } else {
        constexpr int PER = (ROWS + 7) / 8;
        const bool ok = col0 + lane < ncol;
        float v[PER];
        #pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int r = warp + 8 * k;
            v[k] = ok && r < ROWS ? in[offs<AX>(col0 + lane, wrap(g0 + r, n_in), b, d0, d1, n_in)] : 0.f;
        }
        #pragma unroll
        for (int k = 0; k < PER; ++k)
            if (warp + 8 * k < ROWS) S[warp + 8 * k][lane] = v[k];
    }
}

/* Write the four outputs acc[m] of column `lane` at positions a0 + 4 warp + m along AX. */
template <int AX, int OUT, bool ACC>
__device__ __forceinline__ void emit(float (*S)[kMlPad], const float acc[4], float* __restrict__ out,
                                     float* __restrict__ out_lo, int a0, int n_out, int col0, int ncol, int b,
                                     int d0, int d1, long long out_elems, int* status)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto put = [&](long long i, float v) {
        if (!USR_IN_BOUNDS(i, out_elems, status)) return;
        if (OUT == 0) {
            out[i] = ACC ? out[i] + v : v;
        } else {   // TF32 hi / lo pair for the tensor-core passes
            const float h = tf32_rna(v);
            out[i] = h;
            out_lo[i] = v - h;
        }
    };
    if (AX == 0) {
        // transpose through shared memory so that each warp writes a line's outputs contiguously
        __syncthreads();
        #pragma unroll
        for (int m = 0; m < 4; ++m) S[4 * warp + m][lane] = acc[m];
        __syncthreads();
        for (int l = warp; l < 32; l += 8)
            if (col0 + l < ncol && a0 + lane < n_out) put(offs<0>(col0 + l, a0 + lane, b, d0, d1, n_out), S[lane][l]);
    } else {
        if (col0 + lane >= ncol) return;
        #pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int o = a0 + 4 * warp + m;
            if (o < n_out) put(offs<AX>(col0 + lane, o, b, d0, d1, n_out), acc[m]);
        }
    }
}

/* CTA coordinates: blockIdx.x = column tile, blockIdx.y = output tile along AX, blockIdx.z = batch index. */
template <int AX, int OUT>
__global__ void __launch_bounds__(256) k_ml_restrict(const float* __restrict__ in, float* __restrict__ out,
                                                     float* __restrict__ out_lo, int d0, int d1, int ncol,
                                                     int n_in, MlTaps taps, long long out_elems, int* status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    __shared__ float S[kMlWinR][kMlPad];
    const int n_out = n_in / 2;
    const int col0 = blockIdx.x * 32, a0 = blockIdx.y * kMlCh, b = blockIdx.z;
    // outputs a0 .. a0 + 31 read fine rows 2 a0 - T .. 2 (a0 + 31) + T
    stage<AX, kMlWinR>(S, in, 2 * a0 - kMlT, n_in, col0, ncol, b, d0, d1);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    // output 4 warp + m takes rows 2 (4 warp + m) + t, t = 0 .. 2T
    #pragma unroll
    for (int r = 0; r < 2 * 3 + 2 * kMlT + 1; ++r) {
        const float v = S[8 * warp + r][lane];
        #pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int t = r - 2 * m;
            if (t >= 0 && t <= 2 * kMlT) acc[m] = fmaf(taps.w[AX][t], v, acc[m]);
        }
    }
    emit<AX, OUT, false>(S, acc, out, out_lo, a0, n_out, col0, ncol, b, d0, d1, out_elems, status);
}

template <int AX, bool ACC>
__global__ void __launch_bounds__(256) k_ml_prolong(const float* __restrict__ in, float* __restrict__ out, int d0,
                                                    int d1, int ncol, int n_in, MlTaps taps, long long out_elems,
                                                    int* status)
{
    pdl_wait();   // the predecessor on this stream has completed (programmatic launch)
    static_assert(kMlWinP <= kMlCh, "the window fits the transpose buffer");
    __shared__ float S[kMlCh][kMlPad];
    const int n_out = 2 * n_in;
    const int col0 = blockIdx.x * 32, a0 = blockIdx.y * kMlCh, b = blockIdx.z;
    // fine outputs a0 .. a0 + 31 (a0 even) read coarse rows a0 / 2 - T / 2 .. a0 / 2 + 15 + T / 2
    const int G0 = a0 / 2 - kMlT / 2;
    stage<AX, kMlWinP>(S, in, G0, n_in, col0, ncol, b, d0, d1);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    // fine o = a0 + 4 warp + m, coarse row G0 + 2 warp + q: tap o - 2 G + T = m - 2 q + 2 T
    #pragma unroll
    for (int q = 0; q < kMlT + 2; ++q) {
        const float v = S[2 * warp + q][lane];
        #pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int t = m - 2 * q + 2 * kMlT;
            if (t >= 0 && t <= 2 * kMlT) acc[m] = fmaf(taps.w[AX][t], v, acc[m]);
        }
    }
    emit<AX, 0, ACC>(S, acc, out, nullptr, a0, n_out, col0, ncol, b, d0, d1, out_elems, status);
}

/*
 * Launch shape for a transfer along AX producing an output of dims od[0..2] (x fastest): columns are x
 * (AX = 1, 2) or the od[1] * od[2] lines (AX = 0); the batch index is z (AX = 1) or y (AX = 2).
 */
template <int AX>
void shape(const int* od, dim3* grid, int* ncol)
{
    const int n_out = od[AX];
    *ncol = AX == 0 ? od[1] * od[2] : od[0];
    const int batch = AX == 0 ? 1 : (AX == 1 ? od[2] : od[1]);
    *grid = dim3((unsigned)((*ncol + 31) / 32), (unsigned)((n_out + kMlCh - 1) / kMlCh), (unsigned)batch);
}

template <int AX, int OUT>
void restrict_axis(const float* in, float* out, float* out_lo, const int* od, const MlTaps& w, int* status,
                   cudaStream_t st)
{
    dim3 g;
    int ncol;
    shape<AX>(od, &g, &ncol);
    const long long elems = (long long)od[0] * od[1] * od[2];
    launch_pdl(k_ml_restrict<AX, OUT>, g, 256, 0, st, in, out, out_lo, od[0], od[1], ncol, 2 * od[AX], w, elems,
               status);
}

template <int AX, bool ACC>
void prolong_axis(const float* in, float* out, const int* od, const MlTaps& w, int* status, cudaStream_t st)
{
    dim3 g;
    int ncol;
    shape<AX>(od, &g, &ncol);
    const long long elems = (long long)od[0] * od[1] * od[2];
    launch_pdl(k_ml_prolong<AX, ACC>, g, 256, 0, st, in, out, od[0], od[1], ncol, od[AX] / 2, w, elems, status);
}

}  // namespace

void launch_ml_restrict(const MlArgs& m, const float* rho, float* t1, float* t2, float* rho_c, float* rho_c_lo,
                        int* status, cudaStream_t st)
{
    const int d1[3] = {m.nc[0], m.n[1], m.n[2]};
    const int d2[3] = {m.nc[0], m.nc[1], m.n[2]};
    const int d3[3] = {m.nc[0], m.nc[1], m.nc[2]};
    restrict_axis<0, 0>(rho, t1, nullptr, d1, m.taps, status, st);
    restrict_axis<1, 0>(t1, t2, nullptr, d2, m.taps, status, st);
    if (rho_c_lo)
        restrict_axis<2, 1>(t2, rho_c, rho_c_lo, d3, m.taps, status, st);
    else
        restrict_axis<2, 0>(t2, rho_c, nullptr, d3, m.taps, status, st);
}

void launch_ml_prolong(const MlArgs& m, const float* psi_c, float* t1, float* t2, float* psi, int* status,
                       cudaStream_t st)
{
    const int d1[3] = {m.n[0], m.nc[1], m.nc[2]};
    const int d2[3] = {m.n[0], m.n[1], m.nc[2]};
    const int d3[3] = {m.n[0], m.n[1], m.n[2]};
    prolong_axis<0, false>(psi_c, t1, d1, m.taps, status, st);
    prolong_axis<1, false>(t1, t2, d2, m.taps, status, st);
    prolong_axis<2, true>(t2, psi, d3, m.taps, status, st);
}

}  // namespace usr
