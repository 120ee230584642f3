// Primal and dual energies of a map held in caller-owned device buffers, computed
// without allocating device memory.
//
// Some callers of this library may not allocate device memory at all: a host program
// that has handed the whole GPU to its own allocator (a framework's caching allocator,
// or the fixed device-memory budget of an on-vehicle mapping process) must not call
// cudaMalloc behind that allocator's back, and a latency-critical loop cannot afford the
// device-wide synchronisation that cudaMalloc and cudaFree may cause.  For them this
// file offers one entry point whose only working memory is a file-scope __device__
// array of fixed size (every GPU that loads the library holds it until the process
// exits).  Its size caps the map at DENSER_NOALLOC_MAX_BLOCKS blocks.
//
// The kernels rebuild what the context-based path keeps in its own buffers: a hash of
// the block coordinates, the 12-entry neighbour table, and the Omega bits (w > 0);
// then they reduce the same per-voxel energy terms in FP64 into per-CTA partial sums,
// and one CTA adds those.
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace denser {
namespace {

constexpr int kNaMaxBlocks = DENSER_NOALLOC_MAX_BLOCKS;
constexpr int kNaSlots = 2 * kNaMaxBlocks;  // power of two
constexpr int kNaGrid = 608;                // fixed grid of the energy pass (one partial sum pair per CTA)
constexpr int kNaThreads = 256;
constexpr int kMaxDevices = 64;

// Byte layout of the scratch array.
constexpr size_t kOffKeys = 0;                                            // u64 [kNaSlots]
constexpr size_t kOffVals = kOffKeys + sizeof(unsigned long long) * kNaSlots;  // i32 [kNaSlots]
constexpr size_t kOffNbr = kOffVals + sizeof(int32_t) * kNaSlots;         // i32 [max][12]
constexpr size_t kOffBits = kOffNbr + sizeof(int32_t) * kNeighbours * kNaMaxBlocks;  // u32 [max][16]
constexpr size_t kOffPart = kOffBits + sizeof(uint32_t) * 16 * kNaMaxBlocks;  // f64 [kNaGrid][2]
constexpr size_t kOffFlag = kOffPart + sizeof(double) * 2 * kNaGrid;      // i32 error flag
constexpr size_t kOffOut = kOffFlag + 16;                                 // f64 [2] result for host outputs
constexpr size_t kScratchBytes = ((kOffOut + 2 * sizeof(double) + 255) / 256) * 256;

// The only device memory of this entry point (about 2.2 MB).  Host code must not
// use this name as an address: it reaches the array through cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Scratch {
    unsigned long long* keys;
    int32_t* vals;
    int32_t* nbr;
    uint32_t* bits;
    double* part;
    int32_t* flag;
};

Scratch carve(unsigned char* base) {
    Scratch s;
    s.keys = reinterpret_cast<unsigned long long*>(base + kOffKeys);
    s.vals = reinterpret_cast<int32_t*>(base + kOffVals);
    s.nbr = reinterpret_cast<int32_t*>(base + kOffNbr);
    s.bits = reinterpret_cast<uint32_t*>(base + kOffBits);
    s.part = reinterpret_cast<double*>(base + kOffPart);
    s.flag = reinterpret_cast<int32_t*>(base + kOffFlag);
    return s;
}

__global__ void na_clear_kernel(Scratch s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNaSlots; i += gridDim.x * blockDim.x) s.keys[i] = kEmptyKey;
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.flag = 0;
}

__global__ void na_insert_kernel(Scratch s, const int32_t* __restrict__ coords, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 c = reinterpret_cast<const int4*>(coords)[i];
        if (!key_in_range(c.x, c.y, c.z, c.w)) {
            atomicOr(s.flag, 1);
            continue;
        }
        const unsigned long long key = pack_key(c.x, c.y, c.z, c.w);
        const uint32_t h = hash_key(key);
        bool done = false;
        for (int p = 0; p < kNaSlots && !done; ++p) {
            const uint32_t slot = (h + (uint32_t)p) & (kNaSlots - 1);
            const unsigned long long prev = atomicCAS(s.keys + slot, kEmptyKey, key);
            if (prev == kEmptyKey) {
                s.vals[slot] = i;
                done = true;
            } else if (prev == key) {
                atomicOr(s.flag, 2);  // a coordinate appears twice
                done = true;
            }
        }
    }
}

__device__ int32_t na_lookup(const Scratch& s, unsigned long long key) {
    const uint32_t h = hash_key(key);
    for (int p = 0; p < kNaSlots; ++p) {
        const uint32_t slot = (h + (uint32_t)p) & (kNaSlots - 1);
        const unsigned long long k = s.keys[slot];
        if (k == key) return s.vals[slot];
        if (k == kEmptyKey) return -1;
    }
    return -1;
}

// Neighbour table and Omega bits (one warp per block).
__global__ void na_tables_kernel(Scratch s, const int32_t* __restrict__ coords, const float* __restrict__ w, int n) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int b = warp; b < n; b += nwarps) {
        const int4 c = reinterpret_cast<const int4*>(coords)[b];
        if (lane < kNeighbours) {
            int dx, dy, dz;
            neighbour_offset(lane, &dx, &dy, &dz);
            int32_t idx = -1;
            if (key_in_range(c.x, (long long)c.y + dx, (long long)c.z + dy, (long long)c.w + dz))
                idx = na_lookup(s, pack_key(c.x, c.y + dx, c.z + dy, c.w + dz));
            s.nbr[(size_t)b * kNeighbours + lane] = idx;
        }
        for (int k = 0; k < 16; ++k) {
            const unsigned word = __ballot_sync(0xffffffffu, w[(size_t)b * kBlockVoxels + 32 * k + lane] > 0.0f);
            if (lane == 0) s.bits[(size_t)b * 16 + k] = word;
        }
    }
}

__device__ inline bool na_omega(const Scratch& s, int b, int l) { return (s.bits[(size_t)b * 16 + (l >> 5)] >> (l & 31)) & 1u; }

// Per-voxel energy terms (the same ones the context's energy kernel sums):
//   P: |grad_Omega u|_2 + (lambda/2) w (u - f)^2;  D: -f div p - (div p)^2 / (2 lambda w),
// over voxels in Omega, in FP64; one partial sum pair per CTA.
__global__ void __launch_bounds__(kNaThreads) na_energy_kernel(Scratch s, const float* __restrict__ f,
                                                               const float* __restrict__ w,
                                                               const float* __restrict__ u,
                                                               const float* __restrict__ p, int n, double lam) {
    __shared__ double red[2][kNaThreads / 32];
    const size_t nv = (size_t)n * kBlockVoxels;
    double accP = 0.0, accD = 0.0;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(v / kBlockVoxels), l = (int)(v % kBlockVoxels);
        if (!na_omega(s, b, l)) continue;
        const int lc[3] = {l & 7, (l >> 3) & 7, l >> 6};
        const int step[3] = {1, 8, 64};
        const double u0 = u[v];
        double tv2 = 0.0, dv = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // forward neighbour (edge e_a(v)) and backward neighbour (edge e_a(v - a))
            int bf = b, lf = l + step[a], bb = b, lb = l - step[a];
            if (lc[a] == 7) bf = s.nbr[(size_t)b * kNeighbours + a], lf = l - 7 * step[a];
            if (lc[a] == 0) bb = s.nbr[(size_t)b * kNeighbours + 3 + a], lb = l + 7 * step[a];
            if (bf >= 0 && na_omega(s, bf, lf)) {
                const double g = (double)u[(size_t)bf * kBlockVoxels + lf] - u0;
                tv2 += g * g;
                dv += (double)p[a * nv + v];
            }
            if (bb >= 0 && na_omega(s, bb, lb)) dv -= (double)p[a * nv + (size_t)bb * kBlockVoxels + lb];
        }
        const double fv = f[v], wv = w[v], r = u0 - fv;
        accP += sqrt(tv2) + 0.5 * lam * wv * r * r;
        accD += -fv * dv - dv * dv / (2.0 * lam * wv);
    }
    for (int o = 16; o > 0; o >>= 1) {
        accP += __shfl_xor_sync(0xffffffffu, accP, o);
        accD += __shfl_xor_sync(0xffffffffu, accD, o);
    }
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = accP, red[1][threadIdx.x >> 5] = accD;
    __syncthreads();
    if (threadIdx.x == 0) {
        double P = 0.0, D = 0.0;
        for (int i = 0; i < kNaThreads / 32; ++i) P += red[0][i], D += red[1][i];
        s.part[2 * blockIdx.x] = P;
        s.part[2 * blockIdx.x + 1] = D;
    }
}

// Adds the partial sums into out[0..1] (NaN when the coordinates were invalid).
__global__ void __launch_bounds__(1024) na_final_kernel(Scratch s, double* out) {
    __shared__ double rp[1024], rd[1024];
    double P = 0.0, D = 0.0;
    for (int i = threadIdx.x; i < kNaGrid; i += blockDim.x) P += s.part[2 * i], D += s.part[2 * i + 1];
    rp[threadIdx.x] = P, rd[threadIdx.x] = D;
    __syncthreads();
    for (int sft = blockDim.x / 2; sft > 0; sft >>= 1) {
        if ((int)threadIdx.x < sft) rp[threadIdx.x] += rp[threadIdx.x + sft], rd[threadIdx.x] += rd[threadIdx.x + sft];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool bad = *s.flag != 0;
        out[0] = bad ? nan("") : rp[0];
        out[1] = bad ? nan("") : rd[0];
    }
}

// Per-device address of the scratch array, looked up once per device with that device
// current (the first call on a device does this).
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DENSER_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return DENSER_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return DENSER_OK;
}

// True when p is device (or managed) memory that the current device can dereference:
// device memory of another GPU is rejected, since these kernels read the buffers
// directly and a foreign pointer without peer access would fault instead of failing.
bool on_current_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace
}  // namespace denser

extern "C" int denser_energy_noalloc(const int32_t* coords, const float* f, const float* w, const float* u,
                                     const float* p, int64_t n_blocks, double lambda, double* out, void* stream) {
    using namespace denser;
    if (n_blocks < 0 || !out || !(lambda > 0)) return DENSER_ERR_INVALID_ARG;
    if (n_blocks > kNaMaxBlocks) return DENSER_ERR_TOO_LARGE;
    // an error left pending by an earlier, unrelated runtime call must not be read as
    // this call's launch failure below
    cudaGetLastError();
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DENSER_ERR_CUDA;
    }
    if (n_blocks > 0) {
        // the kernels read coords as int4 and the fields as float: a misaligned pointer
        // would fault on the device, so it is refused here, before any launch
        if (!coords || !f || !w || !u || !p || !aligned(coords, 16) || !aligned(f, 4) || !aligned(w, 4) ||
            !aligned(u, 4) || !aligned(p, 4))
            return DENSER_ERR_INVALID_ARG;
        if (!on_current_device(coords, dev) || !on_current_device(f, dev) || !on_current_device(w, dev) ||
            !on_current_device(u, dev) || !on_current_device(p, dev))
            return DENSER_ERR_INVALID_ARG;
    }
    cudaPointerAttributes oat;
    if (cudaPointerGetAttributes(&oat, out) != cudaSuccess) {
        cudaGetLastError();
        return DENSER_ERR_INVALID_ARG;
    }
    const bool dev_out = oat.type == cudaMemoryTypeDevice || oat.type == cudaMemoryTypeManaged;
    if (dev_out && (!aligned(out, 8) || (oat.type == cudaMemoryTypeDevice && oat.device != dev)))
        return DENSER_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    const Scratch s = carve(base);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)n_blocks;
    na_clear_kernel<<<64, 256, 0, st>>>(s);
    if (n > 0) {
        na_insert_kernel<<<(n + 255) / 256, 256, 0, st>>>(s, coords, n);
        na_tables_kernel<<<(n + 7) / 8, 256, 0, st>>>(s, coords, w, n);
    }
    na_energy_kernel<<<kNaGrid, kNaThreads, 0, st>>>(s, f, w, u, p, n, lambda);
    double* res = dev_out ? out : reinterpret_cast<double*>(base + kOffOut);
    na_final_kernel<<<1, 1024, 0, st>>>(s, res);
    if (cudaGetLastError() != cudaSuccess) return DENSER_ERR_CUDA;
    if (!dev_out) {
        if (cudaMemcpyAsync(out, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return DENSER_ERR_CUDA;
        }
    }
    return DENSER_OK;
}
