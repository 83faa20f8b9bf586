/*
 * usr_internal.h -- internal declarations shared by the libusr translation
 * units: the host-side plan (FP64 set-up of the u-series tables) and the
 * argument structs and launchers of the device kernels.
 */
#pragma once

#include <cstdint>
#include <new>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/usr.h"

namespace usr {

constexpr int kMaxPolyDeg = 24;
constexpr int kMaxExplicit = 8;
constexpr int kMaxTerms = 16;
constexpr int kMaxFullTerms = 4096;   // terms of the full real-space series (down to amplitude 1e-20 c)
constexpr int kMlT = 16;           // multilevel transfer half-width in fine points: ceil(6 x 2.6)
constexpr int kGridMargin = 8;      // grid points per axis required beyond the stencil width
constexpr int kMaxGridAxis = 4096;  // grid points per axis at most (bounds the host tables of a plan)
constexpr long long kMaxGridPoints = (1LL << 31) - 1;   // grid points at most (signed 32-bit headroom)
constexpr int kMaxAtoms = 1 << 28;  // atoms per context at most (32-bit cluster-slot indices keep headroom)
constexpr double kMaxBox = 1.0e5;   // box side at most (Angstrom): the pair kernel's padding rows, at -1e6 A and
                                    // beyond, then stay more than 7e5 A from every atom and periodic image
constexpr int kGridMeanBlocks = 304;   // CTAs of the grid-mean reduction (two per SM)
constexpr int kCombineBlocks = 608;    // CTAs of the near + far combination at most (four per SM)

/*
 * Programmatic dependent launch between consecutive kernels of one stream: a kernel launched with
 * launch_pdl is scheduled as soon as its predecessor has completed, or earlier, once every CTA of the
 * predecessor has run pdl_trigger; it calls pdl_wait, which returns when the predecessor has completed
 * and its writes are visible, before touching anything the predecessor reads or writes.  Only the
 * cell-list kernels before the fork trigger early: their successors' waiting CTAs then hold SM slots
 * nothing else needs, whereas waiting CTAs beside the pair kernel and the far chain slowed both.
 * Without the launch attribute (USR_PDL 0) both calls are no-ops and the launches are ordinary ones.
 */
#ifndef USR_PDL
#define USR_PDL 1
#endif
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = USR_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<P>(args)...);
}
#endif
#ifndef USR_GATHER_THREADS
#define USR_GATHER_THREADS 128
#endif
#ifndef USR_GATHER_BLOCKS
#define USR_GATHER_BLOCKS (8 * 152)   // measured: 4 x 152 slower at 1 M charges, 16 x 152 slower on the slab
#endif
constexpr int kGatherBlocks = USR_GATHER_BLOCKS;   // gather CTAs at most

/*
 * Cell blocks of the spreading / interpolation kernels and their smem tiles.
 * Block b along axis a covers cells [b kb_a, min((b+1) kb_a, nc_a)); its tile
 * spans grid points org_a[b] .. org_a[b] + T_a - 1 (periodic).  The reduction
 * table lists, for every grid index g of axis a, the (block, tile offset)
 * pairs whose tile holds g: red_cnt_a[g] entries at red_pair_a[g * rmax_a].
 */
constexpr int kTileMaxSmem = 112 * 1024;   // bytes per tile: two CTAs per SM
struct TileGeom {
    int kb[3];      // cells per block per axis
    int nbk[3];     // blocks per axis
    int T[3];       // tile extent per axis (grid points); T[0] % 4 == 0
    int rmax[3];    // reduction-table row length per axis
    int ps;         // plane stride of the tile in shared memory (floats, >= T[0] T[1], a multiple of 4), chosen
                    // so that the spread's lanes hit distinct banks
};

/* Device copies of the per-axis tile tables (owned by the context). */
struct TileTabs {
    const int* org[3];
    const int* red_cnt[3];
    const int2* red_pair[3];
};

/* Host plan: everything usr_init derives from usr_params, in FP64. */
struct Plan {
    usr_params p;
    usr_plan_info info;
    double L[3];
    int n[3];
    double h[3];
    double sigma, c, F0;
    double sigma_s;                      // largest spreading width (reported)
    double sigma_sa[3];                  // spreading width per axis
    double wsum;                         // sum of the spreading weights over a stencil
    int P;                               // stencil points per axis
    int N;                               // far Gaussians on the fine grid (all of them unless multilevel)
    std::vector<double> a, s;            // full real-space term table (a_j, s_j)
    // pair kernel: F(u = r^2) = sum_{e < n_explicit} ea_e exp(-u * einv_e) + poly(2u/r_c^2 - 1)
    int n_explicit;
    std::vector<char> expl;              // expl[j]: term j is one of the explicit Gaussians
    double ea[kMaxExplicit], einv[kMaxExplicit];
    int poly_deg;
    double poly[kMaxPolyDeg + 1];
    // far grid: per term j < N, axis a: zero-mean periodised 1D kernel ktil[a][j][d] (d = 0..n-1)
    // and its mean mu[a][j]; scale[j] multiplies the term (applied in the z pass)
    std::vector<double> ktil[3][kMaxTerms];
    double mu[3][kMaxTerms];
    double scale[kMaxTerms];
    // virial: first and second derivatives (in x) of the same periodised kernels, split the same way
    std::vector<double> ktil_d[2][3][kMaxTerms];
    double mu_d[2][3][kMaxTerms];
    // multilevel (usr_params.multilevel): terms N .. N + Nc - 1 on the coarse grid nc = n / 2 (spacing 2 h).
    // Per axis, restriction r(G) = sum_g eR(g - 2G) f(g) and prolongation f(g) = sum_G eP(g - 2G) t(G) with
    // the banded periodised Gaussian weights ml_w[a][t + kMlT], t = -kMlT .. kMlT (the same width both
    // ways); the coarse 1D kernels ktil_c / mu_c and scale_c as for the fine grid.
    int Nc = 0;
    int nc[3];
    std::vector<double> ml_w[3];
    std::vector<double> ktil_c[3][kMaxTerms];
    double mu_c[3][kMaxTerms];
    double scale_c[kMaxTerms];
    int cells[3];
    TileGeom tile;
    std::vector<int> tile_org[3];        // per axis: tile origin of each block
    std::vector<int> red_cnt[3];         // per axis: covering tiles of each grid index
    std::vector<int> red_pair[3];        // per axis: (block, offset) pairs, rmax per grid index
};

/* Build the plan (host only).  Returns USR_OK or an error. */
usr_status make_plan(const usr_params* p, Plan* out);

/*
 * Run f (returning a usr_status) so that no C++ exception crosses the C ABI: a failed host allocation
 * becomes USR_ERR_OOM, anything else USR_ERR_INTERNAL.
 */
template <typename F>
usr_status guard(F&& f)
{
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return USR_ERR_OOM;
    } catch (...) {
        return USR_ERR_INTERNAL;
    }
}

/* Device bytes a context holds for a plan (the buffers of usr_api.cu's configure). */
double plan_device_bytes(const Plan& P);

/* usr_reconfigure with a plan already made (the serving loop plans once per request). */
usr_status reconfigure_with_plan(usr_ctx* c, const Plan& P, cudaStream_t st);

/* Canonical single-precision box constants per axis (see the oracle's predicate). */
struct BoxF {
    float L[3];       // (float)L
    float invL[3];    // (float)(1/L)
    float cs[3];      // (float)(nc / L)
    float gs[3];      // (float)(n / L): grid coordinate scale
    int nc[3];
    int n[3];
};

/*
 * Debug build (USR_DEBUG_BOUNDS defined): the kernels check their computed
 * indices against the sizes of the buffers they address; an index out of
 * range sets bit 16 of the status word (USR_ERR_INTERNAL) and the access is
 * skipped.  In the normal build the checks compile to nothing.
 */
#ifdef USR_DEBUG_BOUNDS
#define USR_IN_BOUNDS(i, n, status) \
    ((long long)(i) >= 0 && (long long)(i) < (long long)(n) ? true : (atomicOr((status), 16), false))
#else
#define USR_IN_BOUNDS(i, n, status) true
#endif

struct NearArgs {
    BoxF box;
    int max_atoms;        // rows of the per-atom buffers (bounds of the debug build)
    int max_clusters;     // clusters the cluster buffers hold
    int max_groups;       // groups the group table holds
    float rc2;            // (float)(r_c^2)
    float two_over_rc2;   // 2 / r_c^2
    int n_explicit;
    float ea[kMaxExplicit];
    float einv[kMaxExplicit];
    float el2[kMaxExplicit];   // -einv log2(e): exp(-u einv) = 2^(u el2)
    float ne2[kMaxExplicit];   // -2 einv: factor of 2 dF/du
    float poly[kMaxPolyDeg + 1];
    // the same with their signs flipped, for the pair kernel's negated form of F (-F and its
    // derivative accumulate with additions only)
    float npoly[kMaxPolyDeg + 1];
    float nea[kMaxExplicit];   // -ea
    float nne2[kMaxExplicit];  // -ne2
    float nd2fac;              // -2 * two_over_rc2: 2 dF/du from d(-F)/ds
};

/*
 * The cell list as the pair kernels read it: 8-slot clusters (paired layout,
 * see k_cluster_build) with their caller-sorted indices (-1 for padding rows),
 * cells, bounding boxes, per-cell padded slot starts, and the groups of
 * consecutive clusters of one cell that one warp of the half-list kernel owns
 * (per-cell group starts, first cluster of each group).
 */
struct ClusterList {
    const float4* cpos;
    const int* cidx;
    const int* ccell;
    const float4* bblo;
    const float4* bbhi;
    const int* pstart;
    const int* gfull;     // per cell: first full group (scan), total at [ncell]
    const int* gpart;     // per cell: its partial group's index after the full ones (scan), total at [ncell]
    const int* gfirst;
};

struct GridArgs {
    BoxF box;
    int max_atoms;        // rows of the per-atom buffers (bounds of the debug build)
    float hh[3];          // h^2 / (2 sigma_s^2): exponent factor per stencil step
    float dfac[3];        // h / sigma_s^2: derivative factor
    float F0;             // self-interaction constant (per-atom potential)
    float wsum;           // sum of the spreading weights over a stencil
    const double* psi_mean;   // grid mean of psi (its k = 0 mode, zero up to rounding)
    double F0d;           // the same in FP64 (self energy)
    TileGeom tg;
    TileTabs tab;
};

struct ConvGemm {
    int M, N, K;
    const float* A; long long lda, a_s1, a_s2;   // A[b1][b2][m][k] = A + b1*a_s1 + b2*a_s2 + m*lda + k
    const float* B; long long ldb, b_s1, b_s2;   // B[b1][b2][k][n]
    float* C; long long ldc, c_s1, c_s2;         // C[b1][b2][m][n]
    int nb2;                                     // batch = b1 * nb2 + b2
    int nsplit; long long c_split;               // column block j = n / nsplit goes to C + j*c_split
    int mode;                                    // 0 none, 1 rowsum(A) * colw[n], 2 sum_k roww[k] B[k][n]
    const float* dcw; long long dcw_s1;          // weights; per-b1 offset dcw_s1
    const double* mean;                          // mode 1: subtract K*mean from the row sums (may be null)
};

/* One pass of the tensor-core convolutions (k_conv_tc.cu). */
constexpr int kConvTcMaxStages = 6;
constexpr size_t kConvTcMaxSmem = 220 * 1024;   // dynamic part; static shared memory needs the rest
struct ConvTcArgs {
    int pass;               // 1 = x, 2 = y, 3 = z
    int lines;              // valid A rows (output lines) per batch
    int a_rows_per_batch;   // A row offset between batches (0: all batches share A)
    int K;                  // contraction length
    int NT;                 // N tile (B rows per tile, multiple of 16, <= 256)
    int cols;               // output columns per tile (the DC column follows them)
    int ntiles;             // N tiles
    int n_out;              // output columns in all
    int nterms, nx, ny, nz;
    int stages;             // TMA ring depth
    int tmem_cols;          // tensor-memory columns allocated (power of two >= NT)
    int smem;               // dynamic shared memory per CTA (bytes; padded so that the CTAs an SM
                            // can hold never ask for more than 512 TMEM columns together)
    const float* mu;        // per-term mean of the 1D kernel (passes 1, 2)
    void* out_hi;           // pass output (hi part; FP32 psi for pass 3)
    void* out_lo;           // pass output (lo part; unused for pass 3)
    int* status;
    unsigned long long inject_wait_ns;   // tests: > 0 makes the pass wait that long on a barrier nothing completes
    long long out_elems;    // elements of the pass output (bounds of the debug build)
};
/* Inputs of the device-side table build (k_tables.cu). */
struct ConvTableArgs {
    int N, n[3], nmax;
    const double* ktil;     // [3][N][nmax]: zero-mean periodised kernel of term j on axis a
    const double* mu;       // [3][N]: its mean
    const double* scale;    // [N]: term scale (folded into the z tables)
};

struct ConvTcMaps {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

/* Grid transfers of the multilevel far part (k_multilevel.cu): fine n, coarse nc = n / 2 per axis, banded
   weights w[a][t + kMlT] for t = -kMlT .. kMlT (passed by value: constant-bank operands). */
struct MlTaps {
    float w[3][2 * kMlT + 1];
};
struct MlArgs {
    int n[3], nc[3];
    MlTaps taps;
};

// ---- launchers (all enqueue on `st`) ----
/* rho (fine, [z][y][x]) -> rho_c (coarse) through t1 = [n2][n1][nc0], t2 = [n2][nc1][nc0]; with rho_c_lo
   non-null, rho_c / rho_c_lo receive the TF32 hi / lo split of the result (tensor-core coarse passes). */
void launch_ml_restrict(const MlArgs& m, const float* rho, float* t1, float* t2, float* rho_c, float* rho_c_lo,
                        int* status, cudaStream_t st);
/* psi += prolongation of psi_c, through t1 = [nc2][nc1][n0], t2 = [nc2][n1][n0] */
void launch_ml_prolong(const MlArgs& m, const float* psi_c, float* t1, float* t2, float* psi, int* status,
                       cudaStream_t st);
cudaError_t launch_bin(int n, const float4* xyzq, const BoxF& b, int ncell, int* count, int* cell_of, int* slot,
                       float4* wpos, int* cell_start, int* pstart, int* unsorted, int* perm, float4* spos,
                       int* status, cudaStream_t st);
/* The sorted cell list (cell ids, counting sort, per-cell order by caller index); then the pair kernels'
   clusters built from it (they may run on different streams, the second after the first). */
void launch_bin_sorted(int n, const float4* xyzq, const BoxF& b, int ncell, int* count, int* cell_of, int* slot,
                       float4* wpos, int* cell_start, int* pstart, int* gfull, int* gpart, int* queue, int* unsorted,
                       int* perm, float4* spos, int* status, cudaStream_t st);
void launch_clusters(int n, const BoxF& b, int ncell, const int* cell_start, const int* pstart, const int* gfull,
                     const int* gpart, int* gfirst, const float4* spos, int* key, float4* cpos, int* cidx,
                     int* ccell, float4* bblo, float4* bbhi, unsigned long long* near_acc, int max_clusters,
                     int max_groups, int* status, cudaStream_t st);
/* Upper bound of the half-list kernel's groups for n atoms in ncell cells; clusters per group. */
int near_max_groups(int n, int ncell);
int near_group_clusters();
/* Work units (virial slots) of the half-list kernel over max_groups groups; neighbour ranges per group. */
int near_units(int max_groups);
int near_splits();
void launch_near(int max_groups, int deg, const ClusterList& L, const NearArgs& a, int* queue,
                 unsigned long long* acc, double* vir, int* status, int ctas_per_sm, cudaStream_t st);
/* At most ctas_per_sm persistent pair-kernel CTAs per SM for this context (0: as many as fit). */
void set_near_ctas_per_sm(usr_ctx* c, int ctas_per_sm);
void launch_pairs(int max_clusters, const ClusterList& L, const int* perm, const NearArgs& a, int* count,
                  unsigned long long* hash, int* status, cudaStream_t st);
void launch_spread(int P, const float4* spos, const int* cell_start, const GridArgs& g, float* tilebuf, int split,
                   void* rho, void* rho_lo, double* partial, unsigned int* counter, double* mean, int* status,
                   cudaStream_t st, float* rho32 = nullptr);
void launch_grid_dot(const GridArgs& g, const float* a, const float* b, double scale, double* partial,
                     unsigned int* counter, double* out, cudaStream_t st);
void launch_virial_finalize(const double* near_w, const ClusterList& L, int ncell, const double* dots,
                            const double* energy, double* W, cudaStream_t st);
void launch_conv(const ConvGemm& g, int batches, cudaStream_t st);
void launch_fp32_tables(const ConvTableArgs& t, float* Bx, float* Ay, float* Az, float* wx, float* wy, float* wz,
                        cudaStream_t st);
void launch_tc_table(bool bf16, const ConvTableArgs& t, int pass, int batches, const ConvTcArgs& a, void* hi,
                     void* lo, cudaStream_t st);
usr_status make_tmap(CUtensorMap* m, const void* ptr, bool bf16, long long rows, int K, int box_rows);
size_t conv_tc_smem(const ConvTcArgs& g);
usr_status conv_tc_setup(bool bf16, size_t smem);
void launch_conv_tc(bool bf16, const ConvTcMaps& m, const ConvTcArgs& g, int batches, cudaStream_t st);
/* far part at each of the n sorted atoms into far4 (-q grad phi, phi before the k = 0 correction), and psi's
   grid mean into psi_mean through per-CTA sums in partial (kGatherBlocks CTAs at most) and the last CTA */
void launch_gather(int P, int n, const float4* spos, const float* psi, const GridArgs& g, float4* far4,
                   double* partial, unsigned int* counter, double* psi_mean, int* status, cudaStream_t st);
/* near + far in caller order into out (and the parts into near_dbg / far_dbg when non-null); energy[0..3] =
   total, near, far, self and *net_charge = sum q through per-CTA sums in partial (4 per CTA, kCombineBlocks
   CTAs at most) */
void launch_combine(int n, const float4* spos, const int* perm, const unsigned long long* near_acc,
                    const float4* far4, const GridArgs& g, float4* out, float4* near_dbg, float4* far_dbg,
                    double* partial, unsigned int* counter, double* energy, double* net_charge, int* status,
                    cudaStream_t st);
int tile_blocks(const TileGeom& tg);
size_t tile_floats(const TileGeom& tg);
usr_status grid_kernel_setup(size_t smem_bytes);

}  // namespace usr
