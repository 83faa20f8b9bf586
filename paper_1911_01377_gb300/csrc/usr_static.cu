/*
 * usr_static.cu -- usr_cells_static: the cell list of the near part built
 * without any device allocation.
 *
 * Some callers cannot call cudaMalloc at the moment they need a cell list: a
 * host application that hands the GPU a fixed memory pool and forbids every
 * other allocation, code running inside a stream-ordered allocator's
 * callbacks or a CUDA graph being assembled by hand, or a tool injected into
 * another program that must not change its memory footprint.  This entry
 * point serves them: the caller passes the inputs and outputs, and the
 * temporary arrays of the counting sort live in one file-scope device array of
 * fixed size, kStaticBytes, that every GPU which loads the library holds until
 * the process exits.
 *
 * Host code cannot use the array's name as a device address (on the host it
 * names a stand-in object); the first call on each device looks the real
 * address up with cudaGetSymbolAddress, with that device current, and caches
 * it.  That first call should therefore come before any stream capture.
 * Every call shares the array and the array keeps the previous call's
 * contents: the per-cell counters and the status word are cleared on the
 * call's stream before use, and two calls that overlap on the GPU (on
 * different streams, without ordering between them) race on the array.
 */
#include <mutex>

#include "usr_internal.h"

namespace {

constexpr int kStaticMaxAtoms = 1 << 18;     // 262,144 atoms
constexpr int kStaticMaxCells = 1 << 16;     // 65,536 cells
constexpr long long kStaticMaxPerCell = 2048;   // mean atoms per cell (the per-cell sort's shared-memory size)
constexpr int kMaxDevices = 64;

/* Layout of the scratch array (byte offsets, each 256-byte aligned). */
constexpr size_t kOffCount = 0;                                                   // int[kStaticMaxCells]
constexpr size_t kOffPstart = kOffCount + sizeof(int) * kStaticMaxCells;          // int[kStaticMaxCells + 1]
constexpr size_t kOffStatus = kOffPstart + sizeof(int) * (kStaticMaxCells + 64);  // int (padded to 256 B)
constexpr size_t kOffSlot = kOffStatus + 256;                                     // int[kStaticMaxAtoms]
constexpr size_t kOffUnsorted = kOffSlot + sizeof(int) * kStaticMaxAtoms;         // int[kStaticMaxAtoms]
constexpr size_t kOffWpos = kOffUnsorted + sizeof(int) * kStaticMaxAtoms;         // float4[kStaticMaxAtoms]
constexpr size_t kStaticBytes = kOffWpos + sizeof(float4) * kStaticMaxAtoms;      // about 6.3 MB

static_assert(kOffPstart % 256 == 0 && kOffStatus % 256 == 0 && kOffSlot % 256 == 0 &&
              kOffUnsorted % 256 == 0 && kOffWpos % 256 == 0, "scratch sub-arrays must stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_cells_scratch[kStaticBytes];

unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

/* Device address of g_cells_scratch on the current device (looked up once per device). */
usr_status scratch_address(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return USR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cells_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return USR_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return USR_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" usr_status usr_cells_static(int n, const float* xyzq, const double* box, const int* cells, int* cell,
                                       int* perm, int* cell_start, float* xw, void* stream)
{
    if (n < 0 || !box || !cells) return USR_ERR_ARG;
    usr::BoxF b{};
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !(box[a] < 1e30) || cells[a] < 1) return USR_ERR_ARG;
        // each factor is checked before it is multiplied in, so the product (at most 2^32) cannot overflow
        if (cells[a] > kStaticMaxCells) return USR_ERR_CAPACITY;
        ncell *= cells[a];
        if (ncell > kStaticMaxCells) return USR_ERR_CAPACITY;
    }
    if (n > kStaticMaxAtoms) return USR_ERR_CAPACITY;
    // the per-cell sort is quadratic in a cell's occupancy: refuse calls whose mean occupancy already
    // exceeds what one cell's shared-memory sort holds
    if (n > kStaticMaxPerCell * ncell) return USR_ERR_CAPACITY;
    if (!cell_start) return USR_ERR_ARG;
    if (n > 0 && (!xyzq || !aligned16(xyzq) || !cell || !perm || !xw || !aligned16(xw))) return USR_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        b.L[a] = (float)box[a];
        b.invL[a] = (float)(1.0 / box[a]);
        b.cs[a] = (float)((double)cells[a] / box[a]);
        b.gs[a] = 0.0f;
        b.nc[a] = cells[a];
        b.n[a] = 1;
    }
    // a launch error left by earlier, unrelated work on this thread must not be reported as this call's
    cudaGetLastError();
    unsigned char* base = nullptr;
    usr_status s = scratch_address(&base);
    if (s != USR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int* count = reinterpret_cast<int*>(base + kOffCount);
    int* pstart = reinterpret_cast<int*>(base + kOffPstart);
    int* status = reinterpret_cast<int*>(base + kOffStatus);
    int* slot = reinterpret_cast<int*>(base + kOffSlot);
    int* unsorted = reinterpret_cast<int*>(base + kOffUnsorted);
    float4* wpos = reinterpret_cast<float4*>(base + kOffWpos);
    if (n == 0) {
        // every cell empty: cell_start is all zeros
        if (cudaMemsetAsync(cell_start, 0, sizeof(int) * (size_t)(ncell + 1), st) != cudaSuccess) return USR_ERR_CUDA;
        return USR_OK;
    }
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return USR_ERR_CUDA;
    // launch_bin clears the per-cell counters on `st` before counting and returns the first error of its
    // memset and launches
    const cudaError_t e = usr::launch_bin(n, reinterpret_cast<const float4*>(xyzq), b, (int)ncell, count, cell, slot,
                                          wpos, cell_start, pstart, unsorted, perm, reinterpret_cast<float4*>(xw),
                                          status, st);
    return e == cudaSuccess ? USR_OK : USR_ERR_CUDA;
}
