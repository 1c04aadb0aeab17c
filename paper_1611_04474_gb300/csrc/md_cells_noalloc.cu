// md_cells_noalloc.cu -- md_build_cells_noalloc: the cell build without a caller workspace.
//
// Some callers cannot allocate device memory at the point where they bin atoms: code
// running under an allocator that forbids new allocations mid-stream, plugins handed
// only their input and output buffers by a host application, or runtimes that must not
// call cudaMalloc while other work is being recorded.  This entry point serves them.  Its
// scratch (per-atom cell index, per-cell counters, unsorted slots) lives in one
// file-scope device array of fixed size, so the call itself allocates nothing.
//
// The array is part of the loaded module: every GPU that loads this library holds it
// (MD_NOALLOC_SCRATCH_BYTES) until the process exits.  All calls on a device share it
// and it keeps the previous call's contents; the counters are cleared on every call.
// Calls that overlap on the GPU (two streams, or two threads without ordering) race on
// the array and give wrong results: order them on one stream.
#include <mutex>

#include "md_internal.cuh"

namespace mdnb {
namespace {

constexpr size_t kAlignNA = 256;
constexpr size_t align_na(size_t x) { return (x + kAlignNA - 1) & ~(kAlignNA - 1); }

constexpr size_t kOffCellId = 0;
constexpr size_t kOffCellCnt = align_na(sizeof(int32_t) * (size_t)MD_NOALLOC_MAX_ATOMS);
constexpr size_t kOffPermTmp = kOffCellCnt + align_na(sizeof(int32_t) * (size_t)MD_NOALLOC_MAX_CELLS);
constexpr size_t kScratchBytes = kOffPermTmp + align_na(sizeof(int32_t) * (size_t)MD_NOALLOC_MAX_ATOMS);
static_assert(kScratchBytes == MD_NOALLOC_SCRATCH_BYTES, "scratch size in the header is stale");

// The scratch.  In host code this name is only a stand-in for the device symbol; the
// kernels get its device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device and
// kept for the life of the process (not valid after a device reset, which reloads the
// module; the header says so).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace mdnb

using namespace mdnb;

extern "C" int md_build_cells_noalloc(const float *pos_q, const int32_t *type, int32_t n,
                                      const double *box_L, const int32_t *dims,
                                      int32_t *cell_start, int32_t *perm, float *pos_q_sorted,
                                      int32_t *type_sorted, uint32_t *status, void *stream)
{
    if (n < 0 || !box_L || !dims || !cell_start) return MD_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(box_L[d] > 0.0) || !isfinite(box_L[d]) || dims[d] < 1) return MD_ERR_INVALID_ARG;
    long long ncell = (long long)dims[0] * dims[1] * dims[2];
    if (n > MD_NOALLOC_MAX_ATOMS || ncell > MD_NOALLOC_MAX_CELLS) return MD_ERR_TOO_LARGE;
    if (n > 0 && (!pos_q || !type || !perm || !pos_q_sorted || !type_sorted)) return MD_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(pos_q) & 15u) || (reinterpret_cast<uintptr_t>(pos_q_sorted) & 15u))
        return MD_ERR_INVALID_ARG;
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return MD_ERR_CUDA;
    WsLayout ws = {};
    ws.cell_id = kOffCellId;
    ws.cell_cnt = kOffCellCnt;
    ws.perm_tmp = kOffPermTmp;
    ws.total = kScratchBytes;
    BoxF box = make_box(box_L, dims);
    cudaError_t e = launch_build_cells(reinterpret_cast<const float4 *>(pos_q), type, n, box,
                                       cell_start, perm, reinterpret_cast<float4 *>(pos_q_sorted),
                                       type_sorted, ws, static_cast<char *>(base), status,
                                       static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MD_OK : MD_ERR_CUDA;
}
