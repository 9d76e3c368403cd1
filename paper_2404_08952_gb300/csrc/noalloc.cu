// dolinc_rk_step_noalloc: the SSP-RK3 step for callers that cannot allocate device
// memory.  Its workspace is a file-scope device array of fixed size, so the call
// itself allocates nothing.
#include <cuda_runtime.h>

#include <string>

#include "../../include/dolinc.h"

namespace dol {
dolinc_status report_error(dolinc_status s, const std::string &msg);   // api.cu: sets dolinc_last_error
}

namespace {

constexpr size_t kNoAllocBytes = DOLINC_NOALLOC_MAX_BYTES;

// Workspace shared by every call on a device.  In host code this name is only a
// stand-in for the device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

// Device address of the array on the current device.  Looked up at every call (it
// is a table lookup once the module is loaded), so a module reloaded after
// cudaDeviceReset is picked up too.  Returns null and sets *err on failure.
void *device_scratch(std::string *err)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess || !p) {
        *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return nullptr;
    }
    return p;
}

}  // namespace

extern "C" dolinc_status dolinc_rk_step_noalloc(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt,
                                                double *u_dev, dolinc_stream stream)
{
    size_t need = 0;
    dolinc_status st = dolinc_workspace_size(mesh, scheme, &need);
    if (st != DOLINC_OK) return st;
    if (need > kNoAllocBytes)
        return dol::report_error(DOLINC_ERR_INVALID_ARG,
                                 "dolinc_rk_step_noalloc: this mesh and scheme need " + std::to_string(need) +
                                     " bytes of workspace, above the fixed " + std::to_string(kNoAllocBytes) +
                                     " (DOLINC_NOALLOC_MAX_BYTES); use dolinc_rk_step with a caller workspace");
    std::string err;
    void *ws = device_scratch(&err);
    if (!ws) return dol::report_error(DOLINC_ERR_CUDA, "dolinc_rk_step_noalloc: " + err);
    // a fresh workspace, as every other path starts from: the status and barrier words
    st = dolinc_workspace_init(ws, kNoAllocBytes, stream);
    if (st != DOLINC_OK) return st;
    return dolinc_rk_step(mesh, scheme, dt, u_dev, ws, kNoAllocBytes, stream);
}
