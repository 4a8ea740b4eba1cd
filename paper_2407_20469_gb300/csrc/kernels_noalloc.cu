// kernels_noalloc.cu - scratch for the allocation-free Kramers-Kronig entry
// point (apic_kk_spectra_noalloc).
//
// The regular stage takes its per-block scratch grids from the plan's
// workspace. This variant takes them from one fixed array in the module's
// device memory instead, so a call performs no allocation of any kind. The
// array is created when the library is loaded on a device and lives until the
// process exits; every call shares it, so calls that overlap on the GPU race.
// The Kramers-Kronig kernel writes every scratch element before reading it,
// so nothing has to be cleared between calls.
#include <mutex>

#include "internal.cuh"

namespace apic {

namespace {

constexpr size_t kNoAllocBytes = (size_t)8 << 20;                 // 8 MiB
constexpr int kMaxDevices = 64;

// File-scope device array: in host code this name is only a stand-in, never a
// device address; kernels get the address obtained below.
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocBytes / sizeof(float2)];

std::mutex g_mu;
float2* g_addr[kMaxDevices] = {};

}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocBytes; }

// Device address of the static scratch on `device`, which must be current.
// Looked up once per device (cudaGetSymbolAddress), then cached.
cudaError_t noalloc_scratch(int device, float2** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<float2*>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace apic
