// kernels_noalloc.cu - scratch for the allocation-free Kramers-Kronig entry
// point (apic_kk_spectra_noalloc).
//
// The regular stage takes its per-block scratch grids from the plan's
// workspace. This variant takes them from one fixed array in the module's
// device memory instead, so a call performs no allocation of any kind. The
// array's module is loaded (and the array created) by the first address
// look-up on a device, which plan creation does; it lives until the process
// exits. Every call shares it, so calls that overlap on the GPU race. The
// Kramers-Kronig kernel writes every scratch element before reading it, so
// nothing has to be cleared between calls.
#include "internal.cuh""

namespace apic {

namespace {

constexpr size_t kNoAllocBytes = (size_t)8 << 20;                 // 8 MiB

// File-scope device array: in host code this name is only a stand-in, never a
// device address; kernels get the address obtained below.
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocBytes / sizeof(float2)];

}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocBytes; }

// Device address of the static scratch on the current device (`device`, which
// must be current). Looked up on every call rather than cached, so that an
// address never outlives the context it came from (cudaDeviceReset); once the
// module is loaded the look-up allocates nothing.
cudaError_t noalloc_scratch(int device, float2** out) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return e;
    if (cur != device) return cudaErrorInvalidDevice;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<float2*>(p);
    return cudaSuccess;
}

}  // namespace apic
