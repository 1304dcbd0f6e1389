// saq_noalloc.cu -- saq_encode_noalloc: the encode hot path with its scratch
// in a fixed array of the library's device memory, for callers that cannot
// allocate at encode time (see include/saq.h).  The kernels are the ones
// saq_encode launches; only the origin of the scratch differs.
#include <mutex>

#include "saq_internal.h"

namespace {

// 32 MiB of scratch: the projected rows of one call (FP32) and their codes
// during adjustment (one byte each), i.e. 5 bytes per row and kept dimension.
constexpr size_t kScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) float g_noalloc_scratch[kScratchBytes / sizeof(float)];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory; the device address is looked up once per device.
constexpr int kMaxDevices = 128;
std::mutex g_mu;
float *g_scratch_dev[kMaxDevices] = {};

saq_status scratch_address(int dev, float **out) {
    if (dev < 0 || dev >= kMaxDevices)
        return saq::set_error(SAQ_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return saq::set_error(SAQ_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s",
                                  cudaGetErrorString(e));
        g_scratch_dev[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_dev[dev];
    return SAQ_OK;
}

}  // namespace

extern "C" saq_status saq_encode_noalloc(const saq_model *m, const float *X_dev, int64_t n,
                                         uint8_t *codes_dev, float *factors_dev,
                                         void *stream) {
    using namespace saq;
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0) return set_error(SAQ_ERR_INVALID, "n < 0");
    if (n == 0) return SAQ_OK;
    if (!X_dev || !factors_dev || (m->code_bytes > 0 && !codes_dev))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (((uintptr_t)X_dev | (uintptr_t)codes_dev | (uintptr_t)factors_dev) & 15u)
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    int dev = -1;
    SAQ_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev != m->device)
        return set_error(SAQ_ERR_INVALID, "model lives on device %d, current device is %d",
                         m->device, dev);
    cudaStream_t s = (cudaStream_t)stream;
    // a model without kept dimensions needs no scratch, whatever n is
    if (m->dk == 0) return launch_rownorm2(m, X_dev, n, factors_dev, m->nf, s);
    if (encode_scratch_bytes(m, n) > kScratchBytes) {
        int64_t most = 0;
        while (encode_scratch_bytes(m, most + 32) <= kScratchBytes) most += 32;
        return set_error(SAQ_ERR_INVALID,
                         "n = %lld rows x d_kept = %d exceeds the no-allocation scratch of "
                         "%zu bytes (at most %lld rows for this model)",
                         (long long)n, m->dk, kScratchBytes, (long long)most);
    }
    float *O = nullptr;
    saq_status st = scratch_address(dev, &O);
    if (st != SAQ_OK) return st;
    return encode_rows(m, X_dev, n, codes_dev, factors_dev, O, n, s);
}
