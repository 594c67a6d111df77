// mk_noalloc.cu -- fixed scratch for mk_gates_noalloc.
//
// Some callers cannot let a library call cudaMalloc once they are running: a
// serving process that partitions device memory between tenants at start-up
// and forbids any later allocation, or a latency-critical loop where an
// allocation (which may synchronise the device or fail under memory
// pressure) is not acceptable.  mk_gates_noalloc serves them: its scratch
// (gate descriptors and the extracted LWE samples between the blind rotation
// and the key switch) lives in the file-scope device array below, of a fixed
// size, which every GPU that loads the library holds until the process exits.
//
// In host code the symbol g_noalloc_scratch is only a host-side stand-in for
// the device array, not a device address; its device address is obtained with
// cudaGetSymbolAddress, once per device, with that device current.
#include <mutex>

#include "mk_internal.h"

namespace mk {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

}  // namespace

// Device address of the fixed scratch on `device` (which must be current).
// The first call on a device looks the address up; later calls reuse it.
cudaError_t noalloc_scratch(int device, void **ptr) {
    if (device < 0 || device >= kMaxDevices || !ptr) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    }
    *ptr = g_addr[device];
    return cudaSuccess;
}

}  // namespace mk
