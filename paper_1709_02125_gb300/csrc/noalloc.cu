// oc_reduce_noalloc: the row-partial reduction of the executor, for callers that cannot
// allocate device memory.
//
// Some callers run where allocating is not an option: inside a region that is being
// captured into a CUDA graph by someone else, inside an allocator-free real-time or
// safety-critical component, or under a memory pool that must not grow. This entry point
// therefore takes the caller's input and output and keeps its scratch (the per-row
// partials) in one fixed, file-scope device array instead of asking for memory.
//
// The array (kNoAllocMaxPartials doubles, 512 KiB) exists on every GPU that loads the
// library, until the process exits. In host code its name is only a host-side stand-in:
// the device address is obtained once per device with cudaGetSymbolAddress (first call
// on that device, with the device current) and handed to the kernels. Every call shares
// the array: calls whose work overlaps on the GPU (for example on two streams) race on
// it, so callers must order them.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/oc.h"
#include "launch.h"

namespace oc {

namespace {

constexpr long long kNoAllocMaxPartials = 1 << 16;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];
// the reduction mode is read by the kernel from device memory: a constant table of the
// three modes serves as the parameter block
__device__ double g_noalloc_modes[3] = {0.0, 1.0, 2.0};

double* g_partials_addr[kMaxDevices] = {};
double* g_modes_addr[kMaxDevices] = {};

char g_noalloc_err[256] = "";

int noalloc_fail(int code, const char* msg)
{
    strncpy(g_noalloc_err, msg, sizeof(g_noalloc_err) - 1);
    return code;
}

}  // namespace

}  // namespace oc

extern "C" const char* oc_noalloc_last_error(void) { return oc::g_noalloc_err; }

extern "C" int oc_reduce_noalloc(const void* data, int dtype, int rows, int row_len, long long row_pitch,
                                 int op, int mode, double* out, void* stream)
{
    using namespace oc;
    if (!data || !out) return noalloc_fail(OC_ERR_ARG, "oc_reduce_noalloc: null pointer");
    if (dtype != OC_F64 && dtype != OC_F32) return noalloc_fail(OC_ERR_ARG, "oc_reduce_noalloc: dtype");
    if (op < OC_SUM || op > OC_MIN || mode < 0 || mode > 2) return noalloc_fail(OC_ERR_ARG, "oc_reduce_noalloc: op/mode");
    if (rows < 0 || row_len < 0 || row_pitch < row_len) return noalloc_fail(OC_ERR_ARG, "oc_reduce_noalloc: shape");
    const long long chunks = row_len > 0 ? (row_len + 4095) / 4096 : 1;
    const long long n = (long long)rows * chunks;
    if (n > kNoAllocMaxPartials)
        return noalloc_fail(OC_ERR_ARG, "oc_reduce_noalloc: rows * ceil(row_len / 4096) exceeds 65536 partials");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(OC_ERR_CUDA, "oc_reduce_noalloc: no current device");
    if (!g_partials_addr[dev] || !g_modes_addr[dev]) {
        // set-up, once per device, with that device current
        void* p = nullptr;
        void* q = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p ||
            cudaGetSymbolAddress(&q, g_noalloc_modes) != cudaSuccess || !q)
            return noalloc_fail(OC_ERR_CUDA, "oc_reduce_noalloc: cudaGetSymbolAddress failed");
        g_partials_addr[dev] = (double*)p;
        g_modes_addr[dev] = (double*)q;
    }
    double* part = g_partials_addr[dev];
    cudaStream_t st = (cudaStream_t)stream;

    // The same REDUCE launch the executor makes for one 2-D loop over the region, with a
    // view whose slab is the caller's array (no wrap: S = rows).
    LaunchDesc d;
    memset(&d, 0, sizeof(d));
    d.kernel = OC_K_REDUCE;
    d.ndim = 2;
    d.dtype = dtype;
    d.lo[0] = 0; d.hi[0] = row_len;
    d.lo[1] = 0; d.hi[1] = rows;
    d.lo[2] = 0; d.hi[2] = 1;
    d.nargs = 2;
    d.npts[0] = 1;
    d.access[0] = OC_READ;
    d.access[1] = OC_REDUCE;
    DView& v = d.v[0];
    v.base = (char*)data;
    v.row_elems = row_pitch;
    v.pitch = row_pitch;
    v.S = rows > 0 ? rows : 1;
    v.nx = row_len;
    v.ny = 1;
    d.part = part;
    d.part_row0 = 0;
    d.chunks = (int)chunks;
    d.red_op = op;
    d.params = g_modes_addr[dev] + mode;
    d.nparams = 1;
    if (rows > 0 && row_len > 0) {
        cudaError_t e = launch_loop(d, st);
        if (e != cudaSuccess) return noalloc_fail(OC_ERR_CUDA, "oc_reduce_noalloc: reduce launch failed");
    }
    cudaError_t e = launch_combine(part, row_len > 0 ? n : 0, op, out, st);
    if (e != cudaSuccess) return noalloc_fail(OC_ERR_CUDA, "oc_reduce_noalloc: combine launch failed");
    return OC_OK;
}
