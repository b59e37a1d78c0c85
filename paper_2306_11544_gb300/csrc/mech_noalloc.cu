// mech_bin_noalloc: the voxel binning (keys, histogram, prefix sum, ordered
// scatter) for callers that cannot allocate device memory at the point of the
// call -- for example code whose device memory is entirely reserved by
// another allocator (a framework's caching pool that owns the whole GPU), or
// a latency-critical loop where cudaMalloc's implicit device synchronisation
// is not acceptable.  The caller passes device buffers for the inputs and the
// outputs; the working memory (histogram, prefix sums, arrival slots, scatter
// buffer) is a fixed-size array in this library's own device data, which
// every GPU that loads the library holds until the process exits.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "mech.h"
#include "mech_internal.cuh"

namespace mk {

namespace {

constexpr int64_t kNaMaxCells = int64_t(1) << 18;   // 262,144 cells
constexpr int64_t kNaMaxVoxels = int64_t(1) << 19;  // 524,288 voxels
constexpr size_t kNaVpad = ((size_t)kNaMaxVoxels + 1 + kScanTile - 1) / kScanTile * kScanTile;
// word offsets inside the scratch array
constexpr size_t kNaCount = 0;
constexpr size_t kNaStart = kNaVpad;
constexpr size_t kNaBsum = 2 * kNaVpad;
constexpr size_t kNaSlot = kNaBsum + ((kNaVpad / kScanTile + 63) / 64) * 64;
constexpr size_t kNaTmp = kNaSlot + (size_t)kNaMaxCells;
constexpr size_t kNaWords = kNaTmp + (size_t)kNaMaxCells;  // about 6.1 MiB

static __device__ __align__(256) uint32_t g_na_scratch[kNaWords];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
uint32_t* g_na_ptr[kNaMaxDevices] = {};

// Device address of g_na_scratch on the current device, resolved once per
// device.  Host code must not use the symbol itself: on the host it names a
// stand-in object, not device memory.
cudaError_t na_scratch(uint32_t** out, std::string* why) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return e;
    }
    if (dev < 0 || dev >= kNaMaxDevices) {
        *why = "device index beyond the supported range";
        return cudaErrorInvalidDevice;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) {
            *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return e;
        }
        g_na_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

__global__ void k_na_keys(uint32_t n, const double* __restrict__ xyz, double lo0, double lo1, double lo2,
                          double inv_h, int n0, int n1, int n2, uint32_t* __restrict__ count,
                          uint32_t* __restrict__ key, uint32_t* __restrict__ slot) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t base = warp * 32u; base < n; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        const bool valid = i < n;
        uint32_t k = 0;
        if (valid) {
            const int ix = axis_index_f64(xyz[3 * (size_t)i + 0], lo0, inv_h, n0);
            const int iy = axis_index_f64(xyz[3 * (size_t)i + 1], lo1, inv_h, n1);
            const int iz = axis_index_f64(xyz[3 * (size_t)i + 2], lo2, inv_h, n2);
            k = (uint32_t)ix + (uint32_t)n0 * ((uint32_t)iy + (uint32_t)n1 * (uint32_t)iz);
        }
        const uint32_t s = warp_count(count, k, valid);
        if (valid) {
            key[i] = k;
            slot[i] = s;
        }
    }
}

__global__ void k_na_scatter(uint32_t n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ slot,
                             const uint32_t* __restrict__ start, uint32_t* __restrict__ tmp) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        tmp[start[key[i]] + slot[i]] = i;
}

// Cells of a voxel in ascending input index: rank by index inside the voxel.
__global__ void k_na_order(uint32_t n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ start,
                           const uint32_t* __restrict__ tmp, uint32_t* __restrict__ order) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        const uint32_t src = tmp[q];
        const uint32_t k = key[src];
        const uint32_t s = start[k], e = start[k + 1];
        uint32_t rank = 0;
        for (uint32_t t = s; t < e; ++t) rank += (uint32_t)(tmp[t] < src);
        order[s + rank] = src;
    }
}

__global__ void k_na_copy(uint32_t count, const uint32_t* __restrict__ src, uint32_t* __restrict__ dst) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) dst[i] = src[i];
}

}  // namespace

}  // namespace mk

extern "C" int mech_bin_noalloc(int64_t n, const double* xyz, const double lo[3], double voxel,
                                const int32_t dims[3], uint32_t* key, uint32_t* start, uint32_t* order,
                                void* stream) {
    using namespace mk;
    if (n < 0 || n > kNaMaxCells)
        return record_error(MECH_E_ARG, "mech_bin_noalloc: n must be in [0, " + std::to_string(kNaMaxCells) +
                                            "], got " + std::to_string(n));
    if (!lo || !dims || !start || (n > 0 && (!xyz || !key || !order)))
        return record_error(MECH_E_ARG, "mech_bin_noalloc: null pointer argument");
    if (!std::isfinite(voxel) || !(voxel > 0.0) || !std::isfinite(lo[0]) || !std::isfinite(lo[1]) ||
        !std::isfinite(lo[2]))
        return record_error(MECH_E_NONFINITE, "mech_bin_noalloc: voxel must be finite and > 0, lo finite");
    int64_t V = 1;
    for (int d = 0; d < 3; ++d) {
        if (dims[d] < 1) return record_error(MECH_E_ARG, "mech_bin_noalloc: dims must be >= 1");
        V *= dims[d];
        if (V > kNaMaxVoxels)
            return record_error(MECH_E_ARG, "mech_bin_noalloc: grid has more than " + std::to_string(kNaMaxVoxels) +
                                                " voxels, the size of its fixed working memory");
    }
    uint32_t* scratch = nullptr;
    std::string why;
    if (na_scratch(&scratch, &why) != cudaSuccess) return record_error(MECH_E_CUDA, "mech_bin_noalloc: " + why);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t vpad = (uint32_t)(((size_t)V + 1 + kScanTile - 1) / kScanTile * kScanTile);
    uint32_t* count = scratch + kNaCount;
    uint32_t* sstart = scratch + kNaStart;
    uint32_t* bsum = scratch + kNaBsum;
    uint32_t* slot = scratch + kNaSlot;
    uint32_t* tmp = scratch + kNaTmp;
    const uint32_t nn = (uint32_t)n;
    const uint32_t gcap = (uint32_t)device_sms() * 8u;
    const int grid = nn ? (int)std::min<uint32_t>((nn + 255) / 256, gcap) : 1;
    cudaError_t e = launch_zero_u32(count, vpad, s);  // the histogram must start from zero on every call
    if (e == cudaSuccess && nn) {
        k_na_keys<<<grid, 256, 0, s>>>(nn, xyz, lo[0], lo[1], lo[2], 1.0 / voxel, dims[0], dims[1], dims[2], count,
                                        key, slot);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_scan(count, vpad, bsum, sstart, nullptr, nullptr, s);
    if (e == cudaSuccess && nn) {
        k_na_scatter<<<grid, 256, 0, s>>>(nn, key, slot, sstart, tmp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && nn) {
        k_na_order<<<grid, 256, 0, s>>>(nn, key, sstart, tmp, order);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const uint32_t cnt = (uint32_t)V + 1;
        k_na_copy<<<(int)std::min<uint32_t>((cnt + 255) / 256, gcap), 256, 0, s>>>(cnt, sstart, start);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return record_error(MECH_E_CUDA, std::string("mech_bin_noalloc: ") + cudaGetErrorString(e));
    return MECH_OK;
}
