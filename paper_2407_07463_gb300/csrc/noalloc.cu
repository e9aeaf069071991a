// vof_label_noalloc: connected-component tagging of one field without any
// allocation by the library or the caller beyond the input and the output.
//
// The ordinary path (vof_label) needs a context, and a context needs a
// workspace that the caller allocates.  Some callers cannot allocate device
// memory at the moment they need the tags: a plug-in hosted by a framework
// that owns every device allocation and hands it only finished buffers, or
// a real-time loop whose memory budget is fixed at start-up and may not
// grow.  This variant serves them: its scratch (occupancy bits, union-find
// parents, root ranks, block sums) lives in one file-scope device array of
// fixed size that the GPU keeps for as long as the library is loaded.
//
// Limits and rules:
//  - at most kNoAllocMaxCells cells (64^3); larger grids get VOF_ERR_CAPACITY
//    before anything is launched;
//  - the array is shared by every call on a device and keeps the last call's
//    contents: calls whose kernels can overlap on the GPU (other streams,
//    other host threads) race and must be serialised by the caller;
//  - every scratch word a call reads is written earlier in the same call
//    (bits by the packing pass, parents and ranks of occupied cells and
//    roots, every block sum, the count by the scan), so the previous call's
//    contents never leak into a result and nothing needs clearing;
//  - the first call on a device looks the array's device address up with
//    cudaGetSymbolAddress (with that device current); make that first call
//    before starting any stream capture on that device.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kNoAllocMaxCells = 1 << 18;  // 64^3
// worst-case bit words: one per row when nx <= 32, i.e. N words
constexpr size_t kBitsBytes = (size_t)kNoAllocMaxCells * 4;
constexpr size_t kParentBytes = (size_t)kNoAllocMaxCells * 4;
constexpr size_t kRankBytes = (size_t)kNoAllocMaxCells * 4;
constexpr size_t kBlocks = (kNoAllocMaxCells + 1023) / 1024 + 1;
constexpr size_t kBlockBytes = ((kBlocks * 4 + 255) / 256) * 256;
constexpr size_t kOffBits = 0;
constexpr size_t kOffParent = kOffBits + kBitsBytes;
constexpr size_t kOffRank = kOffParent + kParentBytes;
constexpr size_t kOffBtot = kOffRank + kRankBytes;
constexpr size_t kOffBoff = kOffBtot + kBlockBytes;
constexpr size_t kOffCount = kOffBoff + kBlockBytes;
constexpr size_t kScratchBytes = kOffCount + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" vof_status vof_label_noalloc(const void* c_dev, int32_t precision, int32_t nx, int32_t ny,
                                        int32_t nz, double tag_tau, int32_t connectivity, int32_t* label_dev,
                                        int32_t* n_drops_host, void* stream) {
    if (!c_dev || !label_dev || !n_drops_host) return VOF_ERR_ARG;
    if (precision < VOF_FP64 || precision > VOF_MIXED_LEARNED) return VOF_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return VOF_ERR_ARG;
    if (connectivity != 6 && connectivity != 26) return VOF_ERR_ARG;
    if (!(tag_tau >= 0.0 && tag_tau < 1.0)) return VOF_ERR_ARG;
    long long cells = (long long)nx * ny * nz;
    if (cells > kNoAllocMaxCells) return VOF_ERR_CAPACITY;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    unsigned char* s = (unsigned char*)base;
    vof::Dims g = vof::make_dims(nx, ny, nz);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* bits = (uint32_t*)(s + kOffBits);
    int* parent = (int*)(s + kOffParent);
    int* rank = (int*)(s + kOffRank);
    int* btot = (int*)(s + kOffBtot);
    int* boff = (int*)(s + kOffBoff);
    int* count = (int*)(s + kOffCount);
    bool fp64 = precision == VOF_FP64;
    double tau = tag_tau;
    if (!fp64) {
        // float comparison equivalent to (double)c > tau
        float tf = (float)tau;
        if ((double)tf > tau) tf = nextafterf(tf, -1.0f);
        tau = (double)tf;
    }
    if (vof::pack_bits(c_dev, fp64, bits, g, 1, tau, st) != cudaSuccess ||
        vof::label_field(bits, g, connectivity, parent, rank, btot, boff, label_dev, nullptr, 0, count, st,
                         nullptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    int n = 0;
    if (cudaMemcpyAsync(&n, count, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    *n_drops_host = n;
    return VOF_OK;
}
