// cs_codes_noalloc: patches, codes and co-support bitmasks for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (allocation is not a stream operation and breaks the
// capture), applications whose memory is fully owned by another allocator
// (a framework's caching pool, a fixed budget set up at start-up), and
// latency-critical loops where cudaMalloc / cudaFree would synchronise the
// device. For them this entry point computes exactly what cs_codes computes
// without any context and without allocating: its scratch (operator row
// norms, the guard counter and the guard list) is the file-scope device array
// below, of fixed size, which every GPU that loads the library holds until
// the process exits.
#include <mutex>

#include "internal.h"

namespace {

constexpr long long NOALLOC_MAX_PIXELS = 1ll << 20;  // e.g. 1024 x 1024
constexpr int NOALLOC_MAX_K = CS_MAX_K;              // 1024 operator rows
constexpr int NOALLOC_GUARD_CAP = 1 << 20;           // guarded entries per call
constexpr size_t OFF_ROWNORM = 0;                                     // NOALLOC_MAX_K floats
constexpr size_t OFF_COUNT = OFF_ROWNORM + sizeof(float) * NOALLOC_MAX_K;  // guard counter
constexpr size_t OFF_GUARD = OFF_COUNT + 256;                         // guard list
constexpr size_t NOALLOC_BYTES = OFF_GUARD + sizeof(int2) * NOALLOC_GUARD_CAP;  // ~8 MB

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {};

}  // namespace

// The scratch itself. In host code this name is only a host-side stand-in
// for the device symbol, never a device address: the kernels receive the
// address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up, so it should come
// before any stream capture).
static cs_status noalloc_scratch(int device, void** out) {
    if (device < 0 || device >= MAX_DEVICES)
        return cs_set_error(nullptr, CS_ERR_UNSUPPORTED, "cs_codes_noalloc: device %d", device);
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return cs_set_error(nullptr, CS_ERR_CUDA,
                                "cs_codes_noalloc: cannot locate the scratch array on device %d: %s",
                                device, cudaGetErrorString(e));
        }
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return CS_OK;
}

extern "C" cs_status cs_codes_noalloc(const float* img, int H, int W, const float* omega, int k,
                                      const float* mask, const cs_params* prm, float* codes,
                                      float* lead16, uint32_t* bitmask, int32_t* dev_status,
                                      void* stream) {
    const char* fn = "cs_codes_noalloc";
    if (!img || !omega || !mask || !prm || !bitmask || !dev_status)
        return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    if (H < 1 || W < 1 || (long long)H * W > NOALLOC_MAX_PIXELS)
        return cs_set_error(nullptr, CS_ERR_INVALID_ARG,
                            "%s: image %dx%d has more than the %lld pixels its fixed scratch "
                            "supports (use cs_codes)",
                            fn, W, H, NOALLOC_MAX_PIXELS);
    if (k < 1 || k > NOALLOC_MAX_K)
        return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: k=%d outside 1..%d", fn, k,
                            NOALLOC_MAX_K);
    // patch side, tau, patch order and codes form: the checks cs_codes makes
    cs_status s = cs_check_patch(nullptr, fn, prm);
    if (s) return s;
    // the fixed scratch holds no operator operand tiles: FP32 CUDA-core codes only
    if (prm->codes_form == CS_CODES_TC)
        return cs_set_error(nullptr, CS_ERR_UNSUPPORTED, "%s: computes the FP32 codes form only",
                            fn);
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return cs_set_error(nullptr, CS_ERR_CUDA, "%s: no current CUDA device", fn);
    }
    void* base = nullptr;
    s = noalloc_scratch(device, &base);
    if (s) return s;
    unsigned char* scratch = static_cast<unsigned char*>(base);
    cudaStream_t st = (cudaStream_t)stream;
    // the status words start at zero on every call (the guard counter is
    // cleared by the row-norm kernel)
    cudaError_t e = cudaMemsetAsync(dev_status, 0, 2 * sizeof(int32_t), st);
    if (e == cudaSuccess) {
        CodesArgs a{img, H, W, omega, k, mask, prm->p, prm->tau, codes, lead16, bitmask};
        a.order = prm->patch_order;
        a.rownorm = reinterpret_cast<float*>(scratch + OFF_ROWNORM);
        a.guard_count = reinterpret_cast<int*>(scratch + OFF_COUNT);
        a.guard = reinterpret_cast<int2*>(scratch + OFF_GUARD);
        a.guard_cap = NOALLOC_GUARD_CAP;
        a.d_err = dev_status;
        e = launch_codes(a, st);  // FP32 form (a.tc is false)
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess)
        return cs_set_error(nullptr, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return CS_OK;
}
