/*
 * usr_api.cu -- the C ABI of libusr (declared in include/usr.h): context
 * creation (plan + device allocation + table upload), the evaluation
 * sequence on one stream, host-buffer evaluation, status and inspection.
 *
 * Evaluation sequence (one stream, no host synchronisation, no allocation):
 *   bin + sort (cell list) -> near pair kernel (Eq. 20) -> spread ->
 *   x / y / z convolution passes (Sec. V, Eqs. 31-32) -> gather + combine +
 *   FP64 energy reduction.
 */
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>

#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>

#include "usr_internal.h"

using usr::Plan;

// profiling events of one evaluation (stage boundaries on the two streams)
constexpr int kProfEvents = 12;

/* Host-side NVTX range around the enqueueing of one stage (no cost unless a tool is attached). */
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

/* One tensor-core convolution (three passes): split operands (hi, lo), B tables and tensor maps per pass, the
   per-term means of the x and y kernels. */
#ifndef USR_TC_MIN_CTAS
#define USR_TC_MIN_CTAS 0     // split a tensor-core pass into more N tiles below this many CTAs
#endif
#ifndef USR_SIDE_PRIORITY
#define USR_SIDE_PRIORITY 0   // priority of the far chain's stream: 0 highest, 1 default, 2 lowest
#endif
#ifndef USR_NEAR_CTAS
#define USR_NEAR_CTAS 4   // one CTA slot per SM left to the far chain (measured: 5 and 3 slower)
#endif

struct TcConv {
    bool bf16 = false;
    void *rho_hi = nullptr, *rho_lo = nullptr, *X_hi = nullptr, *X_lo = nullptr, *Y_hi = nullptr, *Y_lo = nullptr;
    void* Bt_hi[3] = {nullptr, nullptr, nullptr};
    void* Bt_lo[3] = {nullptr, nullptr, nullptr};
    float* mu = nullptr;
    usr::ConvTcMaps maps[3];
    usr::ConvTcArgs targs[3];
    int tbatches[3] = {0, 0, 0};
};

struct usr_ctx {
    Plan plan;
    int device = 0;
    int max_atoms = 0;
    int ncell = 0;
    long long G = 0;
    usr::BoxF boxf;
    usr::NearArgs near;
    usr::GridArgs grid;
    // cell list
    int *d_count = nullptr, *d_cell_of = nullptr, *d_slot = nullptr, *d_cell_start = nullptr;
    int *d_unsorted = nullptr, *d_perm = nullptr, *d_status = nullptr;
    float4 *d_wpos = nullptr, *d_spos = nullptr;
    unsigned long long* d_nacc = nullptr;   // near part, 4 fixed-point sums per sorted atom
    // 8-atom clusters of the pair kernel (padded layout)
    int max_clusters = 0, max_groups = 0;
    int *d_pstart = nullptr, *d_cidx = nullptr, *d_ccell = nullptr, *d_gfull = nullptr, *d_gpart = nullptr;
    int *d_gfirst = nullptr, *d_queue = nullptr;
    float4 *d_cpos = nullptr, *d_bblo = nullptr, *d_bbhi = nullptr;
    // grids and convolution tables
    float *d_rho = nullptr, *d_X = nullptr, *d_Y = nullptr, *d_psi = nullptr;
    float *d_Bx = nullptr, *d_Ay = nullptr, *d_Az = nullptr, *d_wx = nullptr, *d_wy = nullptr, *d_wz = nullptr;
    double *d_spread_partial = nullptr, *d_mean = nullptr, *d_gather_partial = nullptr, *d_energy = nullptr;
    double* d_netq = nullptr;            // net charge of the last evaluation (FP64)
    unsigned int* d_counters = nullptr;
    double* d_psi_mean = nullptr;
    // spreading tiles and the per-axis tile tables
    float* d_tilebuf = nullptr;
    int* d_tab[3] = {nullptr, nullptr, nullptr};
    // tensor-core convolutions: the fine grid's (TF32x3 or BF16x3) and, with the multilevel form, the coarse
    // grid's (TF32x3)
    bool tc = false, tc_bf16 = false;
    TcConv tcf, tcc;
    double* d_ktab = nullptr;            // 1D kernels, means and scales of the plan (table-build input)
    // virial: per strain component (xx yy zz xy xz yz) FP32 tables {Bx, Ay, Az, wx, wy, wz} and their input
    bool vir = false;
    float* d_vtab[6][6] = {};
    double* d_vktab = nullptr;
    float *d_psiv = nullptr, *d_rho32 = nullptr;
    double *d_vnear = nullptr, *d_vdot = nullptr, *d_vpart = nullptr, *d_W = nullptr;
    bool vir_valid = false;
    // multilevel: the coarse grid's transfers, its FP32 tables (Bx, Ay, Az, wx, wy, wz) and their input, and
    // the scratch of the coarse steps (two transfer buffers, coarse rho, X, Y and psi)
    usr::MlArgs ml{};
    int mlN = 0;
    size_t ml_t1 = 0, ml_t2 = 0;
    double* d_cktab = nullptr;
    float* d_ctab[6] = {};
    float* d_mlbuf = nullptr;
    bool ml_tc = false;            // coarse passes on the tensor cores (else the FP32 tables above)
    // allocated bytes of every device buffer (buffers only grow), and the
    // pinned staging area of the table uploads with the event of its last use
    std::unordered_map<void**, size_t> cap;
    unsigned char* h_stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    // host-buffer staging and inspection
    float4 *d_in = nullptr, *d_out = nullptr, *d_near_dbg = nullptr, *d_far_dbg = nullptr;
    float4* d_far4 = nullptr;      // far part per sorted atom (gather -> combination)
    bool keep_parts = false;
    bool inject_timeout = false;
    int near_ctas_per_sm = USR_NEAR_CTAS;   // persistent pair-kernel CTAs per SM (0: as many as fit)
    bool parts_valid = false;
    // the far chain (spread, convolutions, psi mean) runs on `side`, a high-priority stream forked from and
    // joined back to the caller's stream, while the pair kernel runs on the caller's stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // profiling: stage boundary events (see usr_stage_times)
    int prof = 0;                  // 1: events at every stage boundary, 2: around the pair kernel only
    int prof_valid = 0;
    cudaEvent_t ev[kProfEvents];
    bool ev_made = false;
    cudaStream_t last_stream = nullptr;
    int last_n = 0;
};

namespace {

template <typename T>
usr_status dalloc(T** p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? USR_ERR_OOM : USR_ERR_CUDA;
    }
    return USR_OK;
}

void free_all(usr_ctx* c)
{
    void* ptrs[] = {c->d_count, c->d_cell_of, c->d_slot, c->d_cell_start, c->d_unsorted, c->d_perm, c->d_status,
                    c->d_pstart, c->d_cidx, c->d_ccell, c->d_cpos, c->d_bblo, c->d_bbhi,
                    c->d_wpos, c->d_spos, c->d_nacc, c->d_gfull, c->d_gpart, c->d_gfirst, c->d_queue, c->d_rho, c->d_X, c->d_Y, c->d_psi, c->d_Bx, c->d_Ay,
                    c->d_Az, c->d_wx, c->d_wy, c->d_wz, c->d_spread_partial, c->d_mean, c->d_gather_partial,
                    c->d_energy, c->d_netq, c->d_counters, c->d_in, c->d_out, c->d_near_dbg, c->d_far_dbg, c->d_far4, c->d_tilebuf,
                    c->d_tab[0], c->d_tab[1], c->d_tab[2], c->d_psi_mean, c->d_ktab};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (TcConv* t : {&c->tcf, &c->tcc}) {
        void* tp[] = {t->rho_hi, t->rho_lo, t->X_hi, t->X_lo, t->Y_hi, t->Y_lo, t->Bt_hi[0], t->Bt_hi[1],
                      t->Bt_hi[2], t->Bt_lo[0], t->Bt_lo[1], t->Bt_lo[2], t->mu};
        for (void* p : tp)
            if (p) cudaFree(p);
    }
    void* vptrs[] = {c->d_vktab, c->d_psiv, c->d_rho32, c->d_vnear, c->d_vdot, c->d_vpart, c->d_W,
                     c->d_cktab, c->d_mlbuf};
    for (float* p : c->d_ctab)
        if (p) cudaFree(p);
    for (void* p : vptrs)
        if (p) cudaFree(p);
    for (auto& comp : c->d_vtab)
        for (float* p : comp)
            if (p) cudaFree(p);
    if (c->ev_made)
        for (auto& e : c->ev) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->stage_ev) cudaEventDestroy(c->stage_ev);
    if (c->h_stage) cudaFreeHost(c->h_stage);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

usr_status check_launch()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? USR_OK : USR_ERR_CUDA;
}

void fill_box(const Plan& P, usr::BoxF& b)
{
    for (int a = 0; a < 3; ++a) {
        b.L[a] = (float)P.L[a];
        b.invL[a] = (float)(1.0 / P.L[a]);
        b.cs[a] = (float)((double)P.cells[a] / P.L[a]);
        b.gs[a] = (float)((double)P.n[a] / P.L[a]);
        b.nc[a] = P.cells[a];
        b.n[a] = P.n[a];
    }
}

size_t tab_ints(const Plan& P, int a)
{
    const size_t head = (P.tile_org[a].size() + P.red_cnt[a].size() + 1) / 2 * 2;
    return head + P.red_pair[a].size();
}

/*
 * Tile shape of one tensor-core pass with n_out output columns and contraction K, over `ctas_m` M tiles (lines /
 * 128 x batches).  When that gives fewer than USR_TC_MIN_CTAS CTAs, the columns are split into more N tiles (16
 * columns at least) so that more SMs share the pass.
 */
void tc_shape(usr::ConvTcArgs& a, int n_out, int K, bool bf16, long long ctas_m)
{
    a.n_out = n_out;
    a.K = K;
    a.ntiles = (n_out + 1 + 255) / 256;
    while (ctas_m * a.ntiles < USR_TC_MIN_CTAS && (n_out + a.ntiles) / (a.ntiles + 1) >= 16) ++a.ntiles;
    a.cols = (n_out + a.ntiles - 1) / a.ntiles;
    a.NT = ((a.cols + 1 + 15) / 16) * 16;
    a.tmem_cols = 32;
    while (a.tmem_cols < a.NT) a.tmem_cols *= 2;
    const int kstage = bf16 ? 64 : 32;
    const int nk = (K + kstage - 1) / kstage;
    const size_t stage = (size_t)(2 * 128 + 2 * a.NT) * 128;
    int S = (int)((200 * 1024) / stage);
    S = std::min(S, std::min(nk, 4));
    a.stages = std::max(1, std::min(S, usr::kConvTcMaxStages));
    // keep (CTAs per SM) x (TMEM columns) <= 512 by padding the shared memory request
    const size_t floor_smem = (size_t)228 * 1024 * a.tmem_cols / 512 + 1024;
    a.smem = (int)std::max(usr::conv_tc_smem(a), floor_smem);
}

/* Grow a device buffer to at least `bytes` (contents are not kept; growing synchronises). */
usr_status ensure(usr_ctx* c, void** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    auto it = c->cap.find(p);
    if (it != c->cap.end() && it->second >= bytes && *p) return USR_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        c->cap[p] = 0;
        return e == cudaErrorMemoryAllocation ? USR_ERR_OOM : USR_ERR_CUDA;
    }
    c->cap[p] = bytes;
    return USR_OK;
}

/* Host tables of one configuration, packed for one staged upload. */
struct Staged {
    std::vector<unsigned char> bytes;
    struct Item { void* dst; size_t off, len; };
    std::vector<Item> items;
    template <typename T>
    void add(void* dst, const T* src, size_t count)
    {
        size_t off = (bytes.size() + 255) / 256 * 256;
        bytes.resize(off + sizeof(T) * count);
        std::memcpy(bytes.data() + off, src, sizeof(T) * count);
        items.push_back({dst, off, sizeof(T) * count});
    }
};

void fill_args(usr_ctx* c);

}  // namespace

/* Mirrors the buffer list of configure (sizes in bytes, each at least 16). */
double usr::plan_device_bytes(const Plan& P)
{
    const bool tc = P.p.conv == USR_CONV_TF32X3 || P.p.conv == USR_CONV_BF16X3;
    const double na = P.p.max_atoms > 0 ? P.p.max_atoms : 1;
    const double ncell = (double)P.cells[0] * P.cells[1] * P.cells[2];
    const double G = (double)P.n[0] * P.n[1] * P.n[2], N = P.N;
    const double nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const double nsb = tile_blocks(P.tile);
    const double ncl = std::floor((na + 7 * ncell + 7) / 8);
    const double nmax = std::max(nx, std::max(ny, nz));
    double b = 4096 + 4 * (ncell + 1) * 3 + 16 * ncl * 8 + 4 * ncl * 8 + 4 * ncl + 32 * ncl;   // cells, clusters
    b += 8 * (3 * N * nmax + 4 * N);                                               // 1D kernel tables
    b += na * (4 * 4 + 16 * 7 + 32);                                               // per-atom arrays
    const double ngr = near_max_groups((int)na, (int)ncell);
    b += 8 * (ncell + 1) + 4 * ngr + 4;                                            // pair-kernel groups
    b += 4 * G + 8 * (nsb + kGatherBlocks + 4 * kCombineBlocks) + 8 * 11 + 4 * nsb * tile_floats(P.tile);
    for (int a = 0; a < 3; ++a) b += 4.0 * ((P.tile_org[a].size() + P.red_cnt[a].size() + 1) / 2 * 2 + P.red_pair[a].size());
    if (P.p.virial) {   // six FP32 table sets, their inputs, two FP32 grids, warp slots, FP32 scratch grids
        b += 6 * 4 * N * (nx * nx + ny * ny + nz * nz + nx + ny + nz) + 6 * 8 * (3 * N * nmax + 4 * N);
        b += 8 * G + 48 * near_units((int)ngr) + 8 * (16 + kGridMeanBlocks);
        if (tc) b += 4 * G * (1 + 2 * N);
    }
    if (P.Nc > 0) {   // multilevel: weights, coarse tables and their input, scratch, FP32 rho copy (tensor cores)
        const double Nc = P.Nc, cx = P.nc[0], cy = P.nc[1], cz = P.nc[2], Gc = cx * cy * cz;
        const double cmax = std::max(cx, std::max(cy, cz));
        const bool mtc = tc && P.nc[0] % 4 == 0 && P.nc[1] % 4 == 0 && P.nc[2] % 4 == 0;
        b += 8 * (3 * Nc * cmax + 4 * Nc);
        b += 4 * (std::max(nz * ny * cx, cz * cy * nx) + std::max(nz * cy * cx, cz * ny * nx));
        if (mtc) {   // TF32x3 coarse passes: split operands, B tables, means, coarse psi
            b += 4 * Gc * 2 * (1 + 2 * Nc) + 8 * Nc + 4 * Gc;
            const double n_out[3] = {cx, cy, cz}, K[3] = {cx, cy, Nc * cz}, bat[3] = {Nc, Nc, 1};
            for (int p = 0; p < 3; ++p) {
                const double nt = std::floor((n_out[p] + 1 + 255) / 256);
                const double cols = std::ceil(n_out[p] / nt);
                const double NT = std::ceil((cols + 1) / 16) * 16;
                b += 2 * 4 * bat[p] * nt * NT * K[p];
            }
        } else {
            b += 4 * Nc * (cx * cx + cy * cy + cz * cz + cx + cy + cz) + 4 * Gc * (2 + 2 * Nc);
        }
        if (tc && !P.p.virial) b += 4 * G;
    }
    if (!tc) {
        b += 4 * G * (1 + 2 * N) + 4 * N * (nx * nx + ny * ny + nz * nz + nx + ny + nz);
    } else {
        const double es = P.p.conv == USR_CONV_BF16X3 ? 2 : 4;
        b += es * G * 2 * (1 + 2 * N) + 8 * N;
        const double n_out[3] = {nx, ny, nz}, K[3] = {nx, ny, N * nz}, bat[3] = {N, N, 1};
        for (int p = 0; p < 3; ++p) {
            const double nt = std::floor((n_out[p] + 1 + 255) / 256);
            const double cols = std::ceil(n_out[p] / nt);
            const double NT = std::ceil((cols + 1) / 16) * 16;
            b += 2 * es * bat[p] * nt * NT * K[p];
        }
    }
    return b;
}

namespace {

/*
 * Buffers, tile shapes and tensor maps of a tensor-core convolution of N terms on an nx x ny x nz grid
 * (BF16x3 or TF32x3); its last pass writes FP32 into psi.  mu: the x then the y kernel mean of each term.
 */
usr_status setup_tc(usr_ctx* c, TcConv& t, bool bf, int N, int nx, int ny, int nz, const std::vector<float>& mu,
                    float* psi, Staged& up)
{
    usr_status s = USR_OK;
    const size_t es = bf ? 2 : 4, G = (size_t)nx * ny * nz;
    t.bf16 = bf;
    void** bufs[6] = {&t.rho_hi, &t.rho_lo, &t.X_hi, &t.X_lo, &t.Y_hi, &t.Y_lo};
    for (int b = 0; b < 6; ++b)
        if ((s = ensure(c, bufs[b], es * G * (b < 2 ? 1 : (size_t)N))) != USR_OK) return s;
    if ((s = ensure(c, (void**)&t.mu, sizeof(float) * 2 * N)) != USR_OK) return s;
    up.add(t.mu, mu.data(), mu.size());
    const int n_out[3] = {nx, ny, nz};
    const int Ks[3] = {nx, ny, N * nz};
    const int lines[3] = {ny * nz, nx * nz, ny * nx};
    const int batches[3] = {N, N, 1};
    const long long a_rows[3] = {(long long)ny * nz, (long long)N * nx * nz, (long long)ny * nx};
    for (int ps = 0; ps < 3; ++ps) {
        usr::ConvTcArgs& a = t.targs[ps];
        std::memset(&a, 0, sizeof(a));
        tc_shape(a, n_out[ps], Ks[ps], bf, (long long)((lines[ps] + 127) / 128) * batches[ps]);
        const size_t nB = (size_t)batches[ps] * a.ntiles * a.NT * a.K;
        if ((s = ensure(c, &t.Bt_hi[ps], es * nB)) != USR_OK || (s = ensure(c, &t.Bt_lo[ps], es * nB)) != USR_OK)
            return s;
    }
    void* a_hi[3] = {t.rho_hi, t.X_hi, t.Y_hi};
    void* a_lo[3] = {t.rho_lo, t.X_lo, t.Y_lo};
    void* o_hi[3] = {t.X_hi, t.Y_hi, psi};
    void* o_lo[3] = {t.X_lo, t.Y_lo, nullptr};
    for (int ps = 0; ps < 3; ++ps) {
        usr::ConvTcArgs& a = t.targs[ps];
        a.pass = ps + 1;
        a.lines = lines[ps];
        a.a_rows_per_batch = ps == 1 ? nx * nz : 0;
        a.nterms = N;
        a.nx = nx;
        a.ny = ny;
        a.nz = nz;
        a.mu = ps == 0 ? t.mu : (ps == 1 ? t.mu + N : nullptr);
        a.out_hi = o_hi[ps];
        a.out_lo = o_lo[ps];
        a.status = c->d_status;
        a.out_elems = ps == 2 ? (long long)G : (long long)G * (long long)N;
        t.tbatches[ps] = batches[ps];
        const long long b_rows = (long long)batches[ps] * a.ntiles * a.NT;
        if ((s = usr::make_tmap(&t.maps[ps].a_hi, a_hi[ps], bf, a_rows[ps], a.K, 128)) ||
            (s = usr::make_tmap(&t.maps[ps].a_lo, a_lo[ps], bf, a_rows[ps], a.K, 128)) ||
            (s = usr::make_tmap(&t.maps[ps].b_hi, t.Bt_hi[ps], bf, b_rows, a.K, a.NT)) ||
            (s = usr::make_tmap(&t.maps[ps].b_lo, t.Bt_lo[ps], bf, b_rows, a.K, a.NT)))
            return s;
    }
    return USR_OK;
}

/* Enqueue the three passes of a tensor-core convolution on st (the first may carry the test-only wait). */
template <typename F>
void run_tc(const TcConv& t, bool inject, cudaStream_t st, F after)
{
    for (int p = 0; p < 3; ++p) {
        usr::ConvTcArgs ta = t.targs[p];
        ta.inject_wait_ns = (p == 0 && inject) ? 1000000ull : 0ull;   // 1 ms, one evaluation
        usr::launch_conv_tc(t.bf16, t.maps[p], ta, t.tbatches[p], st);
        after(p);
    }
}

/* The coarse grid's scratch: t1 | t2 | rho_c | X_c | Y_c | psi_c (rho_c, X_c, Y_c only for FP32 passes). */
float* ml_psi_c(usr_ctx* c)
{
    const size_t Gc = (size_t)c->plan.nc[0] * c->plan.nc[1] * c->plan.nc[2];
    return c->d_mlbuf + c->ml_t1 + c->ml_t2 + (c->ml_tc ? 0 : Gc * (1 + 2 * (size_t)c->mlN));
}

/*
 * Make `c` evaluate the system described by p: plan on the host, grow device
 * buffers that are too small, and upload the tables through the pinned
 * staging area with asynchronous copies on `st`.  Buffers already large
 * enough are reused, so reconfiguring among systems of similar size allocates
 * nothing and does not synchronise the device.
 */
usr_status configure_plan(usr_ctx* c, const Plan& np, cudaStream_t st)
{
    usr_status s = USR_OK;
    c->plan = np;
    const usr_params* p = &c->plan.p;
    const Plan& P = c->plan;
    c->max_atoms = p->max_atoms;
    c->ncell = P.cells[0] * P.cells[1] * P.cells[2];
    c->G = (long long)P.n[0] * P.n[1] * P.n[2];
    c->tc = p->conv == USR_CONV_TF32X3 || p->conv == USR_CONV_BF16X3;
    c->tc_bf16 = p->conv == USR_CONV_BF16X3;
    const size_t na = (size_t)(c->max_atoms > 0 ? c->max_atoms : 1);
    const size_t N = (size_t)P.N, G = (size_t)c->G;
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int nsb = usr::tile_blocks(P.tile);
    c->max_clusters = (int)((na + 7 * (size_t)c->ncell + 7) / 8);
    c->max_groups = usr::near_max_groups((int)na, c->ncell);
    const size_t ncl = (size_t)c->max_clusters;
    const size_t f4 = sizeof(float4), i4 = sizeof(int), fl = sizeof(float), db = sizeof(double);
#define ENSURE(ptr, bytes) \
    if ((s = ensure(c, (void**)&(ptr), (bytes))) != USR_OK) return s;
    ENSURE(c->d_count, i4 * c->ncell);
    // the cell counters start at zero; every evaluation's scan leaves them zero again
    if (cudaMemsetAsync(c->d_count, 0, i4 * c->ncell, st) != cudaSuccess) return USR_ERR_CUDA;
    ENSURE(c->d_cell_start, i4 * (c->ncell + 1));
    ENSURE(c->d_pstart, i4 * (c->ncell + 1));
    ENSURE(c->d_cpos, f4 * ncl * 8);
    ENSURE(c->d_cidx, i4 * ncl * 8);
    ENSURE(c->d_ccell, i4 * ncl);
    ENSURE(c->d_gfull, i4 * (c->ncell + 1));
    ENSURE(c->d_gpart, i4 * (c->ncell + 1));
    ENSURE(c->d_queue, i4);
    ENSURE(c->d_gfirst, i4 * c->max_groups);
    ENSURE(c->d_bblo, f4 * ncl);
    ENSURE(c->d_bbhi, f4 * ncl);
    ENSURE(c->d_cell_of, i4 * na);
    ENSURE(c->d_slot, i4 * na);
    ENSURE(c->d_unsorted, i4 * na);
    ENSURE(c->d_perm, i4 * na);
    ENSURE(c->d_status, i4);
    ENSURE(c->d_wpos, f4 * na);
    ENSURE(c->d_spos, f4 * na);
    ENSURE(c->d_nacc, sizeof(unsigned long long) * 4 * na);
    ENSURE(c->d_psi, fl * G);
    ENSURE(c->d_spread_partial, db * nsb);
    ENSURE(c->d_mean, db);
    ENSURE(c->d_gather_partial, db * (usr::kGatherBlocks + 4 * usr::kCombineBlocks));
    ENSURE(c->d_far4, f4 * na);
    ENSURE(c->d_energy, db * 4);
    ENSURE(c->d_netq, db);
    ENSURE(c->d_counters, sizeof(unsigned int) * 8);
    ENSURE(c->d_psi_mean, db);
    ENSURE(c->d_in, f4 * na);
    ENSURE(c->d_out, f4 * na);
    ENSURE(c->d_near_dbg, f4 * na);
    ENSURE(c->d_far_dbg, f4 * na);
    ENSURE(c->d_tilebuf, fl * nsb * usr::tile_floats(P.tile));
    for (int a = 0; a < 3; ++a) ENSURE(c->d_tab[a], i4 * tab_ints(P, a));
    Staged up;
    c->vir = p->virial != 0;
    c->vir_valid = false;
    if (!c->tc || c->vir) {
        ENSURE(c->d_rho, fl * G);
        ENSURE(c->d_X, fl * N * G);
        ENSURE(c->d_Y, fl * N * G);
        ENSURE(c->d_Bx, fl * nx * N * nx);
        ENSURE(c->d_Ay, fl * N * ny * ny);
        ENSURE(c->d_Az, fl * nz * N * nz);
        ENSURE(c->d_wx, fl * N * nx);
        ENSURE(c->d_wy, fl * N * ny);
        ENSURE(c->d_wz, fl * N * nz);
    }
    // 1D kernels of the plan: [3][N][nmax] values, then [3][N] means, then [N] scales
    const int nmax = std::max(nx, std::max(ny, nz));
    const size_t nkt = 3 * N * (size_t)nmax + 3 * N + N;
    ENSURE(c->d_ktab, db * nkt);
    {
        std::vector<double> kt(nkt, 0.0);
        for (int a = 0; a < 3; ++a)
            for (size_t j = 0; j < N; ++j) {
                std::copy(P.ktil[a][j].begin(), P.ktil[a][j].end(), kt.begin() + (a * N + j) * nmax);
                kt[3 * N * nmax + a * N + j] = P.mu[a][j];
            }
        for (size_t j = 0; j < N; ++j) kt[3 * N * nmax + 3 * N + j] = P.scale[j];
        up.add(c->d_ktab, kt.data(), kt.size());
    }
    // virial: per strain component, the 1D kernels with the derivative order of each axis and the
    // term weight scale_j s_j^2 (the s_j^2 d_a d_b of each term's kernel, Eq. 31 separability)
    static const int kVirOrder[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    usr::ConvTableArgs vtab[6];
    if (c->vir) {
        ENSURE(c->d_vktab, db * nkt * 6);
        ENSURE(c->d_psiv, fl * G);
        if (c->tc) ENSURE(c->d_rho32, fl * G);
        ENSURE(c->d_vnear, db * 6 * usr::near_units(c->max_groups));
        ENSURE(c->d_vdot, db * 6);
        ENSURE(c->d_vpart, db * usr::kGridMeanBlocks);
        ENSURE(c->d_W, db * 9);
        for (int cmp = 0; cmp < 6; ++cmp) {
            ENSURE(c->d_vtab[cmp][0], fl * nx * N * nx);
            ENSURE(c->d_vtab[cmp][1], fl * N * ny * ny);
            ENSURE(c->d_vtab[cmp][2], fl * nz * N * nz);
            ENSURE(c->d_vtab[cmp][3], fl * N * nx);
            ENSURE(c->d_vtab[cmp][4], fl * N * ny);
            ENSURE(c->d_vtab[cmp][5], fl * N * nz);
        }
        std::vector<double> kt(nkt * 6, 0.0);
        for (int cmp = 0; cmp < 6; ++cmp) {
            double* base = kt.data() + nkt * cmp;
            for (int a = 0; a < 3; ++a) {
                const int o = kVirOrder[cmp][a];
                for (size_t j = 0; j < N; ++j) {
                    const std::vector<double>& src = o == 0 ? P.ktil[a][j] : P.ktil_d[o - 1][a][j];
                    std::copy(src.begin(), src.end(), base + (a * N + j) * nmax);
                    base[3 * N * nmax + a * N + j] = o == 0 ? P.mu[a][j] : P.mu_d[o - 1][a][j];
                }
            }
            for (size_t j = 0; j < N; ++j) base[3 * N * nmax + 3 * N + j] = P.scale[j] * P.s[j] * P.s[j];
            usr::ConvTableArgs& t = vtab[cmp];
            t.N = (int)N;
            t.n[0] = nx;
            t.n[1] = ny;
            t.n[2] = nz;
            t.nmax = nmax;
            t.ktil = c->d_vktab + nkt * cmp;
            t.mu = t.ktil + 3 * N * nmax;
            t.scale = t.ktil + 3 * N * nmax + 3 * N;
        }
        up.add(c->d_vktab, kt.data(), kt.size());
    }
    // multilevel: transfer weights (FP32, three axes) and the coarse grid's 1D kernels, in the fine layout.
    // With tensor-core fine passes the coarse passes run on the tensor cores too, in TF32x3 whatever the fine
    // form (the wide terms' near-constant parts need more than the 16 bits of BF16x3), when every coarse
    // extent is a multiple of 4 (16-byte rows of the tensor maps); else in FP32.
    usr::ConvTableArgs ctab{};
    c->mlN = P.Nc;
    c->ml_tc = P.Nc > 0 && c->tc && P.nc[0] % 4 == 0 && P.nc[1] % 4 == 0 && P.nc[2] % 4 == 0;
    if (P.Nc > 0) {
        const size_t Nc = (size_t)P.Nc;
        const int cx = P.nc[0], cy = P.nc[1], cz = P.nc[2];
        const size_t Gc = (size_t)cx * cy * cz;
        const int cmax = std::max(cx, std::max(cy, cz));
        for (int a = 0; a < 3; ++a) {
            c->ml.n[a] = P.n[a];
            c->ml.nc[a] = P.nc[a];
            for (int t = 0; t <= 2 * usr::kMlT; ++t) c->ml.taps.w[a][t] = (float)P.ml_w[a][t];
        }
        const size_t nkc = 3 * Nc * (size_t)cmax + 3 * Nc + Nc;
        ENSURE(c->d_cktab, db * nkc);
        std::vector<double> kt(nkc, 0.0);
        for (int a = 0; a < 3; ++a)
            for (size_t j = 0; j < Nc; ++j) {
                std::copy(P.ktil_c[a][j].begin(), P.ktil_c[a][j].end(), kt.begin() + (a * Nc + j) * cmax);
                kt[3 * Nc * cmax + a * Nc + j] = P.mu_c[a][j];
            }
        for (size_t j = 0; j < Nc; ++j) kt[3 * Nc * cmax + 3 * Nc + j] = P.scale_c[j];
        up.add(c->d_cktab, kt.data(), kt.size());
        if (!c->ml_tc) {
            ENSURE(c->d_ctab[0], fl * cx * Nc * cx);
            ENSURE(c->d_ctab[1], fl * Nc * cy * cy);
            ENSURE(c->d_ctab[2], fl * cz * Nc * cz);
            ENSURE(c->d_ctab[3], fl * Nc * cx);
            ENSURE(c->d_ctab[4], fl * Nc * cy);
            ENSURE(c->d_ctab[5], fl * Nc * cz);
        }
        c->ml_t1 = std::max((size_t)nz * ny * cx, (size_t)cz * cy * nx);
        c->ml_t2 = std::max((size_t)nz * cy * cx, (size_t)cz * ny * nx);
        ENSURE(c->d_mlbuf, fl * (c->ml_t1 + c->ml_t2 + (c->ml_tc ? Gc : Gc * (2 + 2 * Nc))));
        if (c->tc) ENSURE(c->d_rho32, fl * G);
        ctab.N = (int)Nc;
        ctab.n[0] = cx;
        ctab.n[1] = cy;
        ctab.n[2] = cz;
        ctab.nmax = cmax;
        ctab.ktil = c->d_cktab;
        ctab.mu = c->d_cktab + 3 * Nc * cmax;
        ctab.scale = c->d_cktab + 3 * Nc * cmax + 3 * Nc;
    }
    usr::ConvTableArgs tab{};
    tab.N = (int)N;
    tab.n[0] = nx;
    tab.n[1] = ny;
    tab.n[2] = nz;
    tab.nmax = nmax;
    tab.ktil = c->d_ktab;
    tab.mu = c->d_ktab + 3 * N * nmax;
    tab.scale = c->d_ktab + 3 * N * nmax + 3 * N;
    fill_args(c);
    // per axis: tile origins, then reduction counts, then (block, offset) pairs
    for (int a = 0; a < 3; ++a) {
        std::vector<int> t;
        t.insert(t.end(), P.tile_org[a].begin(), P.tile_org[a].end());
        t.insert(t.end(), P.red_cnt[a].begin(), P.red_cnt[a].end());
        while (t.size() % 2) t.push_back(0);
        t.insert(t.end(), P.red_pair[a].begin(), P.red_pair[a].end());
        up.add(c->d_tab[a], t.data(), t.size());
        const size_t off_cnt = P.tile_org[a].size();
        const size_t off_pair = (off_cnt + P.red_cnt[a].size() + 1) / 2 * 2;
        c->grid.tab.org[a] = c->d_tab[a];
        c->grid.tab.red_cnt[a] = c->d_tab[a] + off_cnt;
        c->grid.tab.red_pair[a] = reinterpret_cast<const int2*>(c->d_tab[a] + off_pair);
    }
    c->grid.psi_mean = c->d_psi_mean;
    if (c->tc) {
        std::vector<float> mu(2 * N);
        for (size_t j = 0; j < N; ++j) {
            mu[j] = (float)P.mu[0][j];
            mu[N + j] = (float)P.mu[1][j];
        }
        if ((s = setup_tc(c, c->tcf, c->tc_bf16, (int)N, nx, ny, nz, mu, c->d_psi, up)) != USR_OK) return s;
    }
    if (c->ml_tc) {
        const int Nc = P.Nc;
        std::vector<float> mu(2 * Nc);
        for (int j = 0; j < Nc; ++j) {
            mu[j] = (float)P.mu_c[0][j];
            mu[Nc + j] = (float)P.mu_c[1][j];
        }
        if ((s = setup_tc(c, c->tcc, false, Nc, P.nc[0], P.nc[1], P.nc[2], mu, ml_psi_c(c), up)) != USR_OK)
            return s;
    }
#undef ENSURE
    {   // what the context holds (buffers only grow, so this can exceed the plan's own need)
        double held = 0.0;
        for (const auto& kv : c->cap) held += (double)kv.second;
        c->plan.info.device_bytes = held;
    }
    // staged upload: wait until the previous upload has left the staging area
    if (c->stage_ev && cudaEventSynchronize(c->stage_ev) != cudaSuccess) return USR_ERR_CUDA;
    if (up.bytes.size() > c->stage_cap) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->stage_cap = 0;
        if (cudaHostAlloc((void**)&c->h_stage, up.bytes.size(), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return USR_ERR_OOM;
        }
        c->stage_cap = up.bytes.size();
    }
    std::memcpy(c->h_stage, up.bytes.data(), up.bytes.size());
    for (const auto& it : up.items)
        if (cudaMemcpyAsync(it.dst, c->h_stage + it.off, it.len, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return USR_ERR_CUDA;
    if (!c->stage_ev && cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming) != cudaSuccess)
        return USR_ERR_CUDA;
    if (cudaEventRecord(c->stage_ev, st) != cudaSuccess) return USR_ERR_CUDA;
    // convolution tables, built on the device from the uploaded kernels
    if (c->tc) {
        for (int ps = 0; ps < 3; ++ps)
            usr::launch_tc_table(c->tc_bf16, tab, ps + 1, c->tcf.tbatches[ps], c->tcf.targs[ps], c->tcf.Bt_hi[ps],
                                 c->tcf.Bt_lo[ps], st);
    } else {
        usr::launch_fp32_tables(tab, c->d_Bx, c->d_Ay, c->d_Az, c->d_wx, c->d_wy, c->d_wz, st);
    }
    if (c->vir)
        for (int cmp = 0; cmp < 6; ++cmp)
            usr::launch_fp32_tables(vtab[cmp], c->d_vtab[cmp][0], c->d_vtab[cmp][1], c->d_vtab[cmp][2],
                                    c->d_vtab[cmp][3], c->d_vtab[cmp][4], c->d_vtab[cmp][5], st);
    if (c->ml_tc)
        for (int ps = 0; ps < 3; ++ps)
            usr::launch_tc_table(false, ctab, ps + 1, c->tcc.tbatches[ps], c->tcc.targs[ps], c->tcc.Bt_hi[ps],
                                 c->tcc.Bt_lo[ps], st);
    else if (c->mlN > 0)
        usr::launch_fp32_tables(ctab, c->d_ctab[0], c->d_ctab[1], c->d_ctab[2], c->d_ctab[3], c->d_ctab[4],
                                c->d_ctab[5], st);
    return check_launch();
}

usr_status configure(usr_ctx* c, const usr_params* p, cudaStream_t st)
{
    Plan np;
    usr_status s = usr::make_plan(p, &np);
    if (s != USR_OK) return s;
    return configure_plan(c, np, st);
}

void fill_args(usr_ctx* c)
{
    const Plan& P = c->plan;
    fill_box(P, c->boxf);
    usr::NearArgs& a = c->near;
    std::memset(&a, 0, sizeof(a));
    a.box = c->boxf;
    a.max_atoms = c->max_atoms > 0 ? c->max_atoms : 1;
    a.max_clusters = c->max_clusters;
    a.max_groups = c->max_groups;
    a.rc2 = (float)(P.p.r_c * P.p.r_c);
    a.two_over_rc2 = (float)(2.0 / (P.p.r_c * P.p.r_c));
    a.n_explicit = P.n_explicit;
    for (int e = 0; e < P.n_explicit; ++e) {
        a.ea[e] = (float)P.ea[e];
        a.einv[e] = (float)P.einv[e];
        a.el2[e] = (float)(-P.einv[e] * 1.4426950408889634);    // log2(e)
        a.ne2[e] = (float)(-2.0 * P.einv[e]);
    }
    for (int d = 0; d <= usr::kMaxPolyDeg; ++d) {
        a.poly[d] = (float)P.poly[d];
        a.npoly[d] = -a.poly[d];
    }
    for (int e = 0; e < usr::kMaxExplicit; ++e) {
        a.nea[e] = -a.ea[e];
        a.nne2[e] = -a.ne2[e];
    }
    a.nd2fac = -2.0f * a.two_over_rc2;
    usr::GridArgs& g = c->grid;
    std::memset(&g, 0, sizeof(g));
    g.box = c->boxf;
    g.max_atoms = c->max_atoms > 0 ? c->max_atoms : 1;
    for (int ax = 0; ax < 3; ++ax) {
        g.hh[ax] = (float)(P.h[ax] * P.h[ax] / (2.0 * P.sigma_sa[ax] * P.sigma_sa[ax]));
        g.dfac[ax] = (float)(P.h[ax] / (P.sigma_sa[ax] * P.sigma_sa[ax]));
    }
    g.F0 = (float)P.F0;
    g.F0d = P.F0;
    g.wsum = (float)P.wsum;
    g.tg = P.tile;
}

usr_status check_device(const usr_ctx* c)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return USR_ERR_CUDA;
    return dev == c->device ? USR_OK : USR_ERR_ARG;
}

/* Cell list in canonical sorted order (cell ids, counting sort, order by caller index within a cell). */
void bin_sorted(usr_ctx* c, int n, const float4* xyzq, cudaStream_t st)
{
    usr::launch_bin_sorted(n, xyzq, c->boxf, c->ncell, c->d_count, c->d_cell_of, c->d_slot, c->d_wpos,
                           c->d_cell_start, c->d_pstart, c->d_gfull, c->d_gpart, c->d_queue, c->d_unsorted, c->d_perm,
                           c->d_spos, c->d_status, st);
}

/* The pair kernels' 8-atom clusters, groups and zeroed accumulators, from the sorted cell list. */
void build_clusters(usr_ctx* c, int n, cudaStream_t st)
{
    usr::launch_clusters(n, c->boxf, c->ncell, c->d_cell_start, c->d_pstart, c->d_gfull, c->d_gpart, c->d_gfirst,
                         c->d_spos, c->d_slot, c->d_cpos, c->d_cidx, c->d_ccell, c->d_bblo, c->d_bbhi, c->d_nacc,
                         c->max_clusters, c->max_groups, c->d_status, st);
}

void bin_and_cluster(usr_ctx* c, int n, const float4* xyzq, cudaStream_t st)
{
    bin_sorted(c, n, xyzq, st);
    build_clusters(c, n, st);
}

usr::ClusterList cluster_list(const usr_ctx* c)
{
    usr::ClusterList L;
    L.cpos = c->d_cpos;
    L.cidx = c->d_cidx;
    L.ccell = c->d_ccell;
    L.bblo = c->d_bblo;
    L.bbhi = c->d_bbhi;
    L.pstart = c->d_pstart;
    L.gfull = c->d_gfull;
    L.gpart = c->d_gpart;
    L.gfirst = c->d_gfirst;
    return L;
}

/* The evaluation sequence; xyzq/out are device pointers already checked. */
/*
 * The three FP32 convolution passes of Sec. V on rho with the tables
 * {Bx, Ay, Az, wx, wy, wz} into psi (X and Y are the context's scratch); after
 * each pass `after(k)` is called (stage marks).
 */
struct Conv3 {
    int N, nx, ny, nz;
    float *X, *Y;     // scratch of N * nx * ny * nz floats each
};

template <typename F>
void conv3(const Conv3& d, const float* rho, float* const* t, float* psi, cudaStream_t st, F after)
{
    const int N = d.N, nx = d.nx, ny = d.ny, nz = d.nz;
    const long long G = (long long)nx * ny * nz;
    {   // x pass: all terms
        usr::ConvGemm g{};
        g.M = ny * nz; g.N = N * nx; g.K = nx;
        g.A = rho; g.lda = nx;
        g.B = t[0]; g.ldb = (long long)N * nx;
        g.C = d.X; g.ldc = nx;
        g.nb2 = 1; g.nsplit = nx; g.c_split = G;
        g.mode = 1; g.dcw = t[3]; g.mean = nullptr;   // rho has its mean removed already
        usr::launch_conv(g, 1, st);
    }
    after(0);
    {   // y pass: batched over (term, z)
        usr::ConvGemm g{};
        g.M = ny; g.N = nx; g.K = ny;
        g.A = t[1]; g.lda = ny; g.a_s1 = (long long)ny * ny; g.a_s2 = 0;
        g.B = d.X; g.ldb = nx; g.b_s1 = G; g.b_s2 = (long long)ny * nx;
        g.C = d.Y; g.ldc = nx; g.c_s1 = G; g.c_s2 = (long long)ny * nx;
        g.nb2 = nz; g.nsplit = 1 << 30; g.c_split = 0;
        g.mode = 2; g.dcw = t[4]; g.dcw_s1 = ny;
        usr::launch_conv(g, N * nz, st);
    }
    after(1);
    {   // z pass: sum over terms folded into K
        usr::ConvGemm g{};
        g.M = nz; g.N = nx * ny; g.K = N * nz;
        g.A = t[2]; g.lda = (long long)N * nz;
        g.B = d.Y; g.ldb = (long long)nx * ny;
        g.C = psi; g.ldc = (long long)nx * ny;
        g.nb2 = 1; g.nsplit = 1 << 30; g.c_split = 0;
        g.mode = 2; g.dcw = t[5]; g.dcw_s1 = 0;
        usr::launch_conv(g, 1, st);
    }
    after(2);
}

template <typename F>
void fp32_conv(usr_ctx* c, const float* rho, float* const* t, float* psi, cudaStream_t st, F after)
{
    const Plan& P = c->plan;
    conv3(Conv3{P.N, P.n[0], P.n[1], P.n[2], c->d_X, c->d_Y}, rho, t, psi, st, after);
}

/* The evaluation sequence; xyzq/out are device pointers already checked. */
usr_status run_eval(usr_ctx* c, int n, const float4* xyzq, float4* out, double* energy, cudaStream_t st)
{
    const Plan& P = c->plan;
    double* en = energy ? energy : c->d_energy;
    c->last_stream = st;
    c->last_n = n;
    c->parts_valid = false;
    c->prof_valid = false;
    c->vir_valid = false;
    if (n == 0) {
        if (cudaMemsetAsync(en, 0, 4 * sizeof(double), st) != cudaSuccess ||
            cudaMemsetAsync(c->d_netq, 0, sizeof(double), st) != cudaSuccess)
            return USR_ERR_CUDA;
        if (c->vir && cudaMemsetAsync(c->d_W, 0, 9 * sizeof(double), st) != cudaSuccess) return USR_ERR_CUDA;
        c->vir_valid = c->vir;
        return USR_OK;
    }
    // stage boundaries: on the caller's stream 0 start, 1 cell list done, 2 pair kernel done, 9 the
    // combination may start (the far chain joined), 10 end; on the side stream 3 start, 4 spread done, 5-7
    // passes x, y, z done, 8 multilevel coarse steps done, 11 far gather done
    auto mark = [&](int k, cudaStream_t s) {
        if (c->prof == 1 || (c->prof == 2 && (k == 1 || k == 2))) cudaEventRecord(c->ev[k], s);
    };
    NvtxRange r_eval("usr_eval");
    mark(0, st);
    {
        NvtxRange r("usr: cell list");
        bin_sorted(c, n, xyzq, st);
    }
    // fork: the far chain needs only the sorted cell list, so it starts on the side stream while the caller's
    // stream builds the pair kernel's clusters and then runs the pair kernel
    if (cudaEventRecord(c->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(c->side, c->ev_fork, 0) != cudaSuccess)
        return USR_ERR_CUDA;
    {
        NvtxRange r("usr: clusters");
        build_clusters(c, n, st);
    }
    mark(1, st);
    cudaStream_t sd = c->side;
    {
        NvtxRange r("usr: far chain (spread, convolutions, psi mean)");
        mark(3, sd);
        if (c->tc)
            usr::launch_spread(P.P, c->d_spos, c->d_cell_start, c->grid, c->d_tilebuf, c->tc_bf16 ? 2 : 1,
                               c->tcf.rho_hi, c->tcf.rho_lo, c->d_spread_partial, c->d_counters, c->d_mean, c->d_status,
                               sd, (c->vir || c->mlN > 0) ? c->d_rho32 : nullptr);
        else
            usr::launch_spread(P.P, c->d_spos, c->d_cell_start, c->grid, c->d_tilebuf, 0, c->d_rho, nullptr,
                               c->d_spread_partial, c->d_counters, c->d_mean, c->d_status, sd);
        mark(4, sd);
        if (c->tc) {
            run_tc(c->tcf, c->inject_timeout, sd, [&](int k) { mark(5 + k, sd); });
            c->inject_timeout = false;
        } else {
            float* const t[6] = {c->d_Bx, c->d_Ay, c->d_Az, c->d_wx, c->d_wy, c->d_wz};
            fp32_conv(c, c->d_rho, t, c->d_psi, sd, [&](int k) { mark(5 + k, sd); });
        }
        if (c->mlN > 0) {
            // the wide terms on the coarse grid, added to psi (Sec. V, multilevel)
            const Plan& Q = c->plan;
            const size_t Gc = (size_t)Q.nc[0] * Q.nc[1] * Q.nc[2];
            float* t1 = c->d_mlbuf;
            float* t2 = t1 + c->ml_t1;
            float* pc = ml_psi_c(c);
            const float* rho = c->tc ? c->d_rho32 : c->d_rho;
            if (c->ml_tc) {
                usr::launch_ml_restrict(c->ml, rho, t1, t2, static_cast<float*>(c->tcc.rho_hi),
                                        static_cast<float*>(c->tcc.rho_lo), c->d_status, sd);
                run_tc(c->tcc, false, sd, [](int) {});
            } else {
                float* rc = t2 + c->ml_t2;
                float* Xc = rc + Gc;
                float* Yc = Xc + (size_t)c->mlN * Gc;
                usr::launch_ml_restrict(c->ml, rho, t1, t2, rc, nullptr, c->d_status, sd);
                conv3(Conv3{c->mlN, Q.nc[0], Q.nc[1], Q.nc[2], Xc, Yc}, rc, c->d_ctab, pc, sd, [](int) {});
            }
            usr::launch_ml_prolong(c->ml, pc, t1, t2, c->d_psi, c->d_status, sd);
        }
        mark(8, sd);
        usr::launch_gather(P.P, n, c->d_spos, c->d_psi, c->grid, c->d_far4, c->d_gather_partial, c->d_counters + 4,
                           c->d_psi_mean, c->d_status, sd);
        mark(11, sd);
        if (cudaEventRecord(c->ev_join, sd) != cudaSuccess) return USR_ERR_CUDA;
    }
    {
        NvtxRange r("usr: near pairs");
        usr::launch_near(c->max_groups, P.poly_deg, cluster_list(c), c->near, c->d_queue, c->d_nacc,
                         c->vir ? c->d_vnear : nullptr, c->d_status, c->near_ctas_per_sm, st);
        mark(2, st);
    }
    // join
    if (cudaStreamWaitEvent(st, c->ev_join, 0) != cudaSuccess) return USR_ERR_CUDA;
    mark(9, st);
    {
        NvtxRange r("usr: near + far, energy");
        usr::launch_combine(n, c->d_spos, c->d_perm, c->d_nacc, c->d_far4, c->grid, out,
                            c->keep_parts ? c->d_near_dbg : nullptr, c->keep_parts ? c->d_far_dbg : nullptr,
                            c->d_gather_partial + usr::kGatherBlocks, c->d_counters + 1, en, c->d_netq,
                            c->d_status, st);
        mark(10, st);
    }
    if (c->vir) {
        NvtxRange r("usr: virial");
        // far virial: 1/2 <rho, psi_ab> per strain component, then the finalisation with E_far
        const float* rho = c->tc ? c->d_rho32 : c->d_rho;
        for (int cmp = 0; cmp < 6; ++cmp) {
            fp32_conv(c, rho, c->d_vtab[cmp], c->d_psiv, st, [](int) {});
            usr::launch_grid_dot(c->grid, rho, c->d_psiv, 0.5, c->d_vpart, c->d_counters + 3, c->d_vdot + cmp, st);
        }
        usr::launch_virial_finalize(c->d_vnear, cluster_list(c), c->ncell, c->d_vdot, en, c->d_W, st);
    }
    usr_status s = check_launch();
    if (s == USR_OK) {
        c->parts_valid = c->keep_parts;
        c->prof_valid = c->prof;
        c->vir_valid = c->vir;
    }
    return s;
}


}  // namespace

namespace {
usr_status init_ctx(usr_ctx* c, const usr_params* p);
}

extern "C" usr_status usr_init(const usr_params* p, usr_ctx** out)
{
    if (!out) return USR_ERR_ARG;
    *out = nullptr;
    if (!p) return USR_ERR_ARG;
    usr_ctx* c = nullptr;
    try {
        c = new usr_ctx();
    } catch (...) {
        return USR_ERR_OOM;
    }
    // on any error, returned or thrown (a failed host allocation), the partly built context is freed here
    const usr_status s = usr::guard([&] { return init_ctx(c, p); });
    if (s != USR_OK) {
        free_all(c);
        delete c;
        return s;
    }
    *out = c;
    return USR_OK;
}

namespace {

/* The body of usr_init; the caller frees the context when it returns an error. */
usr_status init_ctx(usr_ctx* c, const usr_params* p)
{
    usr_status s = USR_OK;
    {
        Plan probe;
        if ((s = usr::make_plan(p, &probe)) != USR_OK) return s;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        return USR_ERR_CUDA;
    }
    if ((s = usr::grid_kernel_setup(usr::kTileMaxSmem)) != USR_OK) return s;
    if ((s = usr::conv_tc_setup(false, usr::kConvTcMaxSmem)) != USR_OK ||
        (s = usr::conv_tc_setup(true, usr::kConvTcMaxSmem)) != USR_OK)
        return s;
    if ((s = configure(c, p, 0)) != USR_OK) return s;
    if (cudaMemset(c->d_counters, 0, 8 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_energy, 0, 4 * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->d_netq, 0, sizeof(double)) != cudaSuccess)
        return USR_ERR_CUDA;
    for (auto& e : c->ev) cudaEventCreate(&e);
    c->ev_made = true;
    {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking,
                                         USR_SIDE_PRIORITY == 0 ? greatest : (USR_SIDE_PRIORITY == 1 ? 0 : least))
                != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
            return USR_ERR_CUDA;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return USR_ERR_CUDA;
    return USR_OK;
}

}  // namespace

void usr::set_near_ctas_per_sm(usr_ctx* c, int ctas_per_sm)
{
    if (c) c->near_ctas_per_sm = ctas_per_sm > 0 ? ctas_per_sm : 0;
}

usr_status usr::reconfigure_with_plan(usr_ctx* c, const Plan& P, cudaStream_t st)
{
    if (!c) return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    c->parts_valid = false;
    c->prof_valid = false;
    return usr::guard([&] { return configure_plan(c, P, st); });
}

extern "C" usr_status usr_reconfigure(usr_ctx* c, const usr_params* p, void* stream)
{
    if (!c || !p) return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    c->parts_valid = false;
    c->prof_valid = false;
    return usr::guard([&] { return configure(c, p, (cudaStream_t)stream); });
}

extern "C" void usr_destroy(usr_ctx* c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

extern "C" usr_status usr_info(const usr_ctx* c, usr_plan_info* out)
{
    if (!c || !out) return USR_ERR_ARG;
    *out = c->plan.info;
    return USR_OK;
}

extern "C" usr_status usr_eval(usr_ctx* c, int n, const float* xyzq, float* out, double* energy, void* stream)
{
    if (!c || n < 0) return USR_ERR_ARG;
    if (n > c->max_atoms) return USR_ERR_CAPACITY;
    if (n > 0 && (!xyzq || !out || !aligned16(xyzq) || !aligned16(out))) return USR_ERR_ARG;
    if (energy && ((uintptr_t)energy & 7u)) return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    return run_eval(c, n, (const float4*)xyzq, (float4*)out, energy, (cudaStream_t)stream);
}

extern "C" usr_status usr_eval_host(usr_ctx* c, int n, const float* xyzq, float* out, double* energy, void* stream)
{
    if (!c || n < 0) return USR_ERR_ARG;
    if (n > c->max_atoms) return USR_ERR_CAPACITY;
    if (n > 0 && (!xyzq || !out)) return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (n > 0 && cudaMemcpyAsync(c->d_in, xyzq, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return USR_ERR_CUDA;
    s = run_eval(c, n, c->d_in, c->d_out, c->d_energy, st);
    if (s != USR_OK) return s;
    if (n > 0 && cudaMemcpyAsync(out, c->d_out, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return USR_ERR_CUDA;
    if (energy && cudaMemcpyAsync(energy, c->d_energy, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return USR_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? USR_OK : USR_ERR_CUDA;
}

extern "C" usr_status usr_eval_host_async(usr_ctx* c, int n, const float* xyzq, float* out, double* energy,
                                         void* stream)
{
    if (!c || n < 0) return USR_ERR_ARG;
    if (n > c->max_atoms) return USR_ERR_CAPACITY;
    if (n > 0 && (!xyzq || !out)) return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (n > 0 && cudaMemcpyAsync(c->d_in, xyzq, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return USR_ERR_CUDA;
    s = run_eval(c, n, c->d_in, c->d_out, c->d_energy, st);
    if (s != USR_OK) return s;
    if (n > 0 && cudaMemcpyAsync(out, c->d_out, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return USR_ERR_CUDA;
    if (energy && cudaMemcpyAsync(energy, c->d_energy, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return USR_ERR_CUDA;
    return USR_OK;
}

extern "C" usr_status usr_last_device_status(usr_ctx* c)
{
    if (!c) return USR_ERR_ARG;
    if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) return USR_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return USR_ERR_CUDA;
    if (cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) return USR_ERR_CUDA;
    if (v & 9) return USR_ERR_NONFINITE;
    if (v & 4) return USR_ERR_TIMEOUT;
    return (v & 18) ? USR_ERR_INTERNAL : USR_OK;
}

extern "C" usr_status usr_debug_cells(usr_ctx* c, int n, const float* xyzq, int* cell, int* perm, int* cell_start,
                                      float* xw, void* stream)
{
    if (!c || n < 0 || n > c->max_atoms) return USR_ERR_ARG;
    if (n > 0 && (!xyzq || !aligned16(xyzq) || !cell || !perm || !cell_start || !xw || !aligned16(xw)))
        return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    if (n == 0) return USR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    bin_and_cluster(c, n, (const float4*)xyzq, st);
    cudaMemcpyAsync(cell, c->d_cell_of, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(perm, c->d_perm, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(cell_start, c->d_cell_start, sizeof(int) * ((size_t)c->ncell + 1), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(xw, c->d_spos, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    return check_launch();
}

extern "C" usr_status usr_debug_pairs(usr_ctx* c, int n, const float* xyzq, int* count, uint64_t* hash, void* stream)
{
    if (!c || n < 0 || n > c->max_atoms) return USR_ERR_ARG;
    if (n > 0 && (!xyzq || !aligned16(xyzq) || !count || !hash)) return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    if (n == 0) return USR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    bin_and_cluster(c, n, (const float4*)xyzq, st);
    usr::launch_pairs(c->max_clusters, cluster_list(c), c->d_perm, c->near, count, (unsigned long long*)hash,
                      c->d_status, st);
    return check_launch();
}

extern "C" usr_status usr_virial(usr_ctx* c, double* W, void* stream)
{
    if (!c || !W || !c->vir || !c->vir_valid) return USR_ERR_ARG;
    if (cudaMemcpyAsync(W, c->d_W, 9 * sizeof(double), cudaMemcpyDefault, (cudaStream_t)stream) != cudaSuccess)
        return USR_ERR_CUDA;
    return USR_OK;
}

extern "C" usr_status usr_net_charge(usr_ctx* c, double* q, void* stream)
{
    if (!c || !q) return USR_ERR_ARG;
    usr_status s = check_device(c);
    if (s != USR_OK) return s;
    if (cudaMemcpyAsync(q, c->d_netq, sizeof(double), cudaMemcpyDefault, (cudaStream_t)stream) != cudaSuccess)
        return USR_ERR_CUDA;
    return USR_OK;
}

extern "C" usr_status usr_debug_inject_timeout(usr_ctx* c, int on)
{
    if (!c || !c->tc) return USR_ERR_ARG;
    c->inject_timeout = on != 0;
    return USR_OK;
}

extern "C" usr_status usr_set_keep_parts(usr_ctx* c, int on)
{
    if (!c) return USR_ERR_ARG;
    c->keep_parts = on != 0;
    return USR_OK;
}

extern "C" usr_status usr_debug_parts(usr_ctx* c, float* near_out, float* far_out, void* stream)
{
    if (!c) return USR_ERR_ARG;
    if (!c->parts_valid) return USR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = sizeof(float4) * (size_t)c->last_n;
    if (near_out) cudaMemcpyAsync(near_out, c->d_near_dbg, bytes, cudaMemcpyDeviceToDevice, st);
    if (far_out) cudaMemcpyAsync(far_out, c->d_far_dbg, bytes, cudaMemcpyDeviceToDevice, st);
    return check_launch();
}

extern "C" usr_status usr_set_profiling(usr_ctx* c, int on)
{
    if (!c) return USR_ERR_ARG;
    if (on < 0 || on > 2) return USR_ERR_ARG;
    c->prof = on;
    return USR_OK;
}

extern "C" usr_status usr_stage_times(usr_ctx* c, float* ms)
{
    if (!c || !ms) return USR_ERR_ARG;
    if (!c->prof_valid) return USR_ERR_ARG;
    if (c->prof_valid == 2) {
        // the pair kernel alone; the other stages read 0
        if (cudaEventSynchronize(c->ev[2]) != cudaSuccess) return USR_ERR_CUDA;
        for (int k = 0; k < USR_NSTAGES; ++k) ms[k] = 0.f;
        return cudaEventElapsedTime(&ms[1], c->ev[1], c->ev[2]) == cudaSuccess ? USR_OK : USR_ERR_CUDA;
    }
    if (cudaEventSynchronize(c->ev[10]) != cudaSuccess) return USR_ERR_CUDA;
    // (from, to) event pairs of the stages; the gather stage adds the multilevel coarse steps (if any) and
    // the far gather with psi's mean (11 - 7) to the combination (10 - 9); the wait for the later of the two
    // branches (between 2 or 11 and 9) is in no stage
    static const int from[USR_NSTAGES] = {0, 1, 3, 4, 5, 6, 9}, to[USR_NSTAGES] = {1, 2, 4, 5, 6, 7, 10};
    for (int k = 0; k < USR_NSTAGES; ++k) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->ev[from[k]], c->ev[to[k]]) != cudaSuccess) return USR_ERR_CUDA;
        ms[k] = t;
    }
    float gm = 0.f;
    if (cudaEventElapsedTime(&gm, c->ev[7], c->ev[11]) != cudaSuccess) return USR_ERR_CUDA;
    ms[USR_NSTAGES - 1] += gm;
    return USR_OK;
}
