// Warm-start network: a 4-layer 3^3 convolutional network that maps a fused block and
// its one-voxel halo (10^3 voxels; f and a normalised weight) to a starting point (u,
// p_x, p_y, p_z) of the primal-dual iteration on the block's 8^3 voxels.  The paper has
// no such network; these kernels train and run it.
//
// Every layer is computed as a 16 -> 16 channel 3^3 convolution with zero padding over
// the 10^3 grid (the first layer's 2 input channels and the last layer's 4 output
// channels are zero-padded, and their extra weights stay zero because their gradients
// are zero).  Activations are BF16, channel-last: act[sample][voxel][16], voxel
// v = x + 10 y + 100 z.  Weights are BF16 [27 taps][16 out][16 in], tap = dx + 3 dy +
// 9 dz for the offset (dx - 1, dy - 1, dz - 1).  Products run on the tensor cores as
// implicit GEMMs (BF16 in, FP32 accumulate):
//   forward / data gradient: tcgen05.mma, M = 128 padded voxels, N = 16 channels, K = 16
//                            channels of one tap, accumulated in tensor memory;
//   weight gradient:         mma.sync m16n8k16, M = 16 out channels, N = 8 in channels,
//                            K = 16 voxels.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace denser {
namespace {

constexpr int kC = 16;           // channels of every layer as computed
constexpr int kG = 10;           // grid side: block + halo
constexpr int kGV = 1000;        // voxels per sample
constexpr int kP = 12;           // padded tile side
constexpr int kTiles = 63;       // 16-voxel row tiles covering 1000 voxels (1008)
constexpr int kNetThreads = 128;
constexpr size_t kTileBytes = (size_t)kP * kP * kP * kC * 2;   // 55296

__device__ inline unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void ldsm_x4(unsigned addr, unsigned* r) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ inline void ldsm_x4_t(unsigned addr, unsigned* r) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ inline void mma_bf16(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Padded-tile byte offset of grid voxel (x, y, z) shifted by tap offsets (0..2 each).
__device__ inline int tile_off(int x, int y, int z) { return ((z * kP + y) * kP + x) * (kC * 2); }

// Copies one sample [1000][16] bf16 into the padded tile interior (border stays zero).
__device__ inline void load_tile(char* tile, const __nv_bfloat16* src) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    for (int i = threadIdx.x; i < kGV * 2; i += blockDim.x) {
        const int v = i >> 1, half = i & 1;
        const int x = v % kG, y = (v / kG) % kG, z = v / (kG * kG);
        *reinterpret_cast<uint4*>(tile + tile_off(x + 1, y + 1, z + 1) + half * 16) = __ldg(s + i);
    }
}

// ------------------------------------------------------------------ tcgen05 conv
// The same convolution on the fifth-generation tensor cores.  Per sample, the padded
// 12^3 activation grid sits in shared memory in the canonical K-major layout without
// swizzle: two planes of 16-byte rows, plane h holding channels 8h .. 8h + 7 of every
// padded voxel p = x' + 12 y' + 144 z'.  An M-tile is 128 consecutive padded rows; for tap
// (dx, dy, dz) its A operand is the same two planes read from a start row shifted by
// (dx - 1) + 12 (dy - 1) + 144 (dz - 1), so one shared-memory descriptor per (tile, tap)
// and no data movement.  B (the tap's 16 x 16 weights, K-major) has the same two-plane
// layout.  tcgen05.mma (M 128, N 16, K 16, BF16 in, FP32 out) accumulates the 27 taps of
// each of the 12 tiles in tensor memory (16 columns per tile, 192 of the CTA's 256); one
// thread issues the MMAs and commits them to an mbarrier; the four warps wait for it
// (bounded) and read their 32 TMEM lanes back with tcgen05.ld for bias, ReLU and the
// stores.  The 12 tiles start at padded row 157 (grid voxel (0, 0, 0)) and reach row 1692
// (>= 1570, voxel (9, 9, 9)); with the tap shifts they read rows 0 .. 1849.
constexpr int kTcRows = 1856;                              // staged padded rows (zeros beyond the grid)
constexpr int kTcRow0 = 157;                               // padded row of grid voxel (0, 0, 0)
constexpr int kTcTiles = 12;
constexpr uint32_t kTcPlane = (uint32_t)kTcRows * 16;      // 29696 bytes per A plane
constexpr uint32_t kTcA = 2 * kTcPlane;                    // 59392
constexpr uint32_t kTcTap = 2 * kC * 16;                   // 512 bytes of B per tap (two planes)
constexpr uint32_t kTcB = 27 * kTcTap;                     // 13824
// 100 KB per CTA keeps at most two CTAs on an SM, so their TMEM allocations (256 columns
// each of the SM's 512) never wait for each other
constexpr size_t kTcSmem = 100 * 1024;
static_assert((size_t)kTcA + kTcB <= kTcSmem, "planes and weights exceed the conv's shared memory");
constexpr uint32_t kTcCols = 256;                          // TMEM columns per CTA
constexpr long long kTcWaitLimit = 1ll << 24;              // mbarrier polls before a wait counts as lost
// kind::f16 instruction descriptor: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12
// = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) | ((128u >> 4) << 24);

__device__ int g_tc_timeout;  // set when an MMA completion wait ran out (read by denser_net_check)

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte
// offset (between core matrices adjacent in K), stride-dimension byte offset (between
// 8-row groups), descriptor version 1 at bit 46, no swizzle.
__device__ inline uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ inline void tc_mma(uint32_t d, uint64_t a, uint64_t b, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}

__device__ inline bool tc_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ inline void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kNetThreads, 1) conv3_tc_kernel(const __nv_bfloat16* __restrict__ x,
                                                                  const __nv_bfloat16* __restrict__ w,
                                                                  const float* __restrict__ bias, int relu,
                                                                  __nv_bfloat16* __restrict__ y_bf16,
                                                                  float* __restrict__ y_f32, int n) {
    extern __shared__ __align__(128) char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    char* planes = smem;
    char* wts = smem + kTcA;
    for (int i = t; i < (int)(kTcA / 16); i += blockDim.x) reinterpret_cast<uint4*>(planes)[i] = make_uint4(0, 0, 0, 0);
    // weights [tap][co][ci] -> [tap][plane h][co][ci 8h .. 8h + 7]
    for (int i = t; i < 27 * kC * 2; i += blockDim.x) {
        const int tap = i / (kC * 2), co = (i / 2) % kC, h = i & 1;
        *reinterpret_cast<uint4*>(wts + tap * kTcTap + h * (kC * 16) + co * 16) = __ldg(reinterpret_cast<const uint4*>(w) + i);
    }
    float bv[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) bv[c] = bias ? bias[c] : 0.0f;
    const uint32_t bar_a = smem_u32(&bar);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t a0 = smem_u32(planes), b0 = smem_u32(wts);
    uint32_t parity = 0;
    bool lost = false;
    for (int s = blockIdx.x; s < n && !lost; s += gridDim.x) {
        // the sample's voxels into their padded rows (the border rows stay zero)
        const uint4* src = reinterpret_cast<const uint4*>(x + (size_t)s * kGV * kC);
        for (int i = t; i < kGV * 2; i += blockDim.x) {
            const int v = i >> 1, h = i & 1;
            const int px = v % kG + 1, py = (v / kG) % kG + 1, pz = v / (kG * kG) + 1;
            *reinterpret_cast<uint4*>(planes + h * kTcPlane + (px + 12 * py + 144 * pz) * 16) = __ldg(src + i);
        }
        // generic-proxy stores become visible to the tensor cores' async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int tile = 0; tile < kTcTiles; ++tile) {
                const int row0 = kTcRow0 + 128 * tile;
                for (int tap = 0; tap < 27; ++tap) {
                    const int off = (tap % 3 - 1) + 12 * ((tap / 3) % 3 - 1) + 144 * (tap / 9 - 1);
                    const uint64_t ad = tc_desc(a0 + (uint32_t)(row0 + off) * 16, kTcPlane, 128);
                    const uint64_t bd = tc_desc(b0 + (uint32_t)tap * kTcTap, kC * 16, 128);
                    tc_mma(tmem + (uint32_t)(kC * tile), ad, bd, tap > 0);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_a)
                         : "memory");
        }
        long long it = 0;
        bool done = false;
        while (!(done = tc_try_wait(bar_a, parity)) && ++it < kTcWaitLimit) {
        }
        if (!done) {
            if (t == 0) atomicExch(&g_tc_timeout, 1);
            lost = true;
        } else {
            parity ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // warp w reads TMEM lanes 32 w .. 32 w + 31: rows row0 + 32 w + lane of each tile
            for (int tile = 0; tile < kTcTiles; ++tile) {
                float v[kC];
                tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(kC * tile), v);
                const int row = kTcRow0 + 128 * tile + 32 * warp + lane;
                const int px = row % 12, py = (row / 12) % 12, pz = row / 144;
                if (px < 1 || px > kG || py < 1 || py > kG || pz < 1 || pz > kG) continue;
                const int vox = (px - 1) + kG * (py - 1) + kG * kG * (pz - 1);
#pragma unroll
                for (int c = 0; c < kC; ++c) {
                    v[c] += bv[c];
                    if (relu) v[c] = fmaxf(v[c], 0.0f);
                }
                const size_t off = ((size_t)s * kGV + vox) * kC;
                if (y_f32) {
                    float4* d = reinterpret_cast<float4*>(y_f32 + off);
#pragma unroll
                    for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                if (y_bf16) {
                    __nv_bfloat162* d = reinterpret_cast<__nv_bfloat162*>(y_bf16 + off);
#pragma unroll
                    for (int q = 0; q < kC / 2; ++q) d[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();  // TMEM reads and the planes are done before the next sample
    }
    if (lost) {
        // give the MMAs in flight a second bounded chance to land before TMEM is freed
        long long it = 0;
        while (!tc_try_wait(bar_a, parity) && ++it < kTcWaitLimit) {
        }
        __syncthreads();
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// dW[tap][co][ci] += sum_samples sum_v dz[v][co] h[v + offset(tap)][ci] (zero padding);
// db[co] += sum dz[v][co].  Each warp owns taps warp, warp + 4, ... and accumulates them
// over all of the CTA's samples before one atomic flush.
__global__ void __launch_bounds__(kNetThreads) wgrad_kernel(const __nv_bfloat16* __restrict__ h,
                                                             const __nv_bfloat16* __restrict__ dz, float* dw,
                                                             float* db, int n) {
    extern __shared__ __align__(16) char smem[];
    char* tile = smem;                       // padded h
    char* dzs = smem + kTileBytes;           // dz rows [1008][16], rows >= 1000 zero
    __shared__ float dbs[kC];
    for (int i = threadIdx.x; i < (int)(kTileBytes / 16); i += blockDim.x)
        reinterpret_cast<uint4*>(tile)[i] = make_uint4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < kTiles * 16 * 2; i += blockDim.x)
        reinterpret_cast<uint4*>(dzs)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x < kC) dbs[threadIdx.x] = 0.0f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[7][2][4];
#pragma unroll
    for (int q = 0; q < 7; ++q)
        for (int j = 0; j < 2; ++j)
            for (int e = 0; e < 4; ++e) acc[q][j][e] = 0.0f;
    float bsum = 0.0f;  // thread t < 128 sums channel t % 16 over rows t / 16 + 8 i
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        __syncthreads();
        load_tile(tile, h + (size_t)s * kGV * kC);
        const uint4* src = reinterpret_cast<const uint4*>(dz + (size_t)s * kGV * kC);
        for (int i = threadIdx.x; i < kGV * 2; i += blockDim.x) reinterpret_cast<uint4*>(dzs)[i] = __ldg(src + i);
        __syncthreads();
        {
            const __nv_bfloat16* d = reinterpret_cast<const __nv_bfloat16*>(dzs);
            for (int v = threadIdx.x >> 4; v < kGV; v += kNetThreads / 16)
                bsum += __bfloat162float(d[v * kC + (threadIdx.x & 15)]);
        }
        for (int ks = 0; ks < kTiles; ++ks) {
            // A = dz^T (16 co x 16 voxels): rows of dz are voxels; .trans gives the co-major fragment
            const int mtx = lane >> 3, r = lane & 7;
            unsigned a[4];
            {
                const int v = ks * 16 + r + ((mtx >> 1) & 1) * 8;   // matrices: (v0-7,co0-7) (v0-7,co8-15) (v8-15,co0-7) (v8-15,co8-15)
                const int co = (mtx & 1) * 8;
                ldsm_x4_t(smem_u32(dzs) + v * kC * 2 + co * 2, a);
            }
            const int vb = min(ks * 16 + r + (mtx & 1) * 8, kGV - 1);   // B rows: voxels, clamped (dz is zero there)
            const int xb = vb % kG, yb = (vb / kG) % kG, zb = vb / (kG * kG);
            const unsigned brow = smem_u32(tile) + tile_off(xb, yb, zb) + (mtx >> 1) * 16;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const int tap = warp + 4 * q;
                if (tap < 27) {
                    const int dx = tap % 3, dy = (tap / 3) % 3, dzz = tap / 9;
                    unsigned b[4];  // (v0-7, ci0-7) (v8-15, ci0-7) (v0-7, ci8-15) (v8-15, ci8-15)
                    ldsm_x4_t(brow + tile_off(dx, dy, dzz), b);
                    mma_bf16(acc[q][0], a, b[0], b[1]);
                    mma_bf16(acc[q][1], a, b[2], b[3]);
                }
            }
        }
    }
    // flush: fragment (row co = g (+8), cols ci = 8 j + 2 c (+1))
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const int tap = warp + 4 * q;
        if (tap >= 27) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j)
            for (int e = 0; e < 4; ++e) {
                const int co = g + 8 * (e >> 1), ci = 8 * j + 2 * c + (e & 1);
                atomicAdd(dw + (tap * kC + co) * kC + ci, acc[q][j][e]);
            }
    }
    atomicAdd(&dbs[threadIdx.x & 15], bsum);
    __syncthreads();
    if (threadIdx.x < kC) atomicAdd(db + threadIdx.x, dbs[threadIdx.x]);
}

__global__ void relu_backward_kernel(const __nv_bfloat16* __restrict__ dh, const __nv_bfloat16* __restrict__ h,
                                     __nv_bfloat16* __restrict__ dz, long long count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        dz[i] = __bfloat162float(h[i]) > 0.0f ? dh[i] : __float2bfloat16(0.0f);
}

// Masked squared error on the centre 8^3 of channels 0..3; dout (bf16, zero elsewhere)
// = 2 (out - target) mask / n; the loss sum goes to *loss (FP64).
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ target,
                            const float* __restrict__ mask, __nv_bfloat16* __restrict__ dout, double* loss, int n) {
    double acc = 0.0;
    const long long total = (long long)n * kGV;
    const float inv_n = 1.0f / (float)n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / kGV), v = (int)(i % kGV);
        const int x = v % kG, y = (v / kG) % kG, z = v / (kG * kG);
        const bool centre = x >= 1 && x <= 8 && y >= 1 && y <= 8 && z >= 1 && z <= 8;
        float g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (centre) {
            const int l = (x - 1) + 8 * (y - 1) + 64 * (z - 1);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const size_t ti = ((size_t)s * 4 + ch) * 512 + l;
                const float d = (out[i * kC + ch] - target[ti]) * mask[ti];
                acc += (double)d * d;
                g[ch] = 2.0f * d * mask[ti] * inv_n;
            }
        }
        __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(dout + i * kC);
        dst[0] = __floats2bfloat162_rn(g[0], g[1]);
        dst[1] = __floats2bfloat162_rn(g[2], g[3]);
#pragma unroll
        for (int q = 2; q < kC / 2; ++q) dst[q] = __floats2bfloat162_rn(0.0f, 0.0f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / n);
}

__global__ void adam_kernel(float* w, const float* grad, float* m, float* v, int count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gr;
        const float vi = b2 * v[i] + (1.0f - b2) * gr * gr;
        m[i] = mi, v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of FP32 weights [27][16 out][16 in]: the forward layout, and the layout of
// the data-gradient convolution (taps mirrored, in/out swapped).
__global__ void pack_weights_kernel(const float* w32, __nv_bfloat16* wf, __nv_bfloat16* wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * kC * kC; i += gridDim.x * blockDim.x) {
        const int tap = i / (kC * kC), co = (i / kC) % kC, ci = i % kC;
        const __nv_bfloat16 v = __float2bfloat16(w32[i]);
        wf[i] = v;
        wb[((26 - tap) * kC + ci) * kC + co] = v;
    }
}

// ---------------------------------------------------------- map <-> samples
// Network inputs of listed blocks: f and w / (w + 8) on the 10^3 grid of the block and its
// one-voxel halo (all 26 neighbours, found through the hash table), zero elsewhere.
__global__ void gather_kernel(DeviceMap m, const int32_t* __restrict__ blocks, int n, __nv_bfloat16* x) {
    __shared__ int nb27[27];
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        const int b = blocks ? blocks[s] : s;
        __syncthreads();
        if (threadIdx.x < 27) {
            const int4 k = reinterpret_cast<const int4*>(m.coords)[b];
            const int dx = threadIdx.x % 3 - 1, dy = (threadIdx.x / 3) % 3 - 1, dz = threadIdx.x / 9 - 1;
            int idx = -1;
            if (key_in_range(k.x, (long long)k.y + dx, (long long)k.z + dy, (long long)k.w + dz))
                idx = hash_lookup(m, pack_key(k.x, k.y + dx, k.z + dy, k.w + dz));
            nb27[threadIdx.x] = idx;
        }
        __syncthreads();
        for (int v = threadIdx.x; v < kGV; v += blockDim.x) {
            const int gx = v % kG - 1, gy = (v / kG) % kG - 1, gz = v / (kG * kG) - 1;  // -1..8
            const int ox = gx < 0 ? -1 : (gx > 7 ? 1 : 0), oy = gy < 0 ? -1 : (gy > 7 ? 1 : 0),
                      oz = gz < 0 ? -1 : (gz > 7 ? 1 : 0);
            const int nbi = nb27[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)];
            float fv = 0.0f, wn = 0.0f;
            if (nbi >= 0) {
                const int l = (gx - 8 * ox) + 8 * (gy - 8 * oy) + 64 * (gz - 8 * oz);
                const float wv = m.w[(size_t)nbi * kBlockVoxels + l];
                fv = wv > 0.0f ? m.f[(size_t)nbi * kBlockVoxels + l] : 0.0f;
                wn = wv / (wv + 8.0f);
            }
            __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(x + ((size_t)s * kGV + v) * kC);
            dst[0] = __floats2bfloat162_rn(fv, wn);
#pragma unroll
            for (int q = 1; q < kC / 2; ++q) dst[q] = __floats2bfloat162_rn(0.0f, 0.0f);
        }
    }
}

__device__ inline bool omega_of(const DeviceMap& m, int b, int l) {
    return (m.omega_bits[(size_t)b * 16 + (l >> 5)] >> (l & 31)) & 1u;
}

// Edge mask of Eq. 3 at voxel l of block b along axis a: l and its +a neighbour in Omega.
__device__ inline bool edge_of(const DeviceMap& m, int b, int l, int a) {
    if (!omega_of(m, b, l)) return false;
    const int lc = a == 0 ? (l & 7) : (a == 1 ? ((l >> 3) & 7) : (l >> 6));
    const int step = a == 0 ? 1 : (a == 1 ? 8 : 64);
    if (lc < 7) return omega_of(m, b, l + step);
    const int nb = m.nbr[(size_t)b * kNeighbours + a];
    return nb >= 0 && omega_of(m, nb, l - 7 * step);
}

template <typename T>
__global__ void targets_kernel(DeviceMap m, const T* u, const T* p, size_t pstride, const int32_t* __restrict__ blocks,
                               int n, float* target, float* mask, float mu, float mp) {
    const long long total = (long long)n * kBlockVoxels;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / kBlockVoxels), l = (int)(i % kBlockVoxels);
        const int b = blocks ? blocks[s] : s;
        const size_t v = (size_t)b * kBlockVoxels + l;
        const bool o = omega_of(m, b, l);
        target[((size_t)s * 4 + 0) * 512 + l] = Store<T>::ld(u + v);
        mask[((size_t)s * 4 + 0) * 512 + l] = o ? mu : 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            target[((size_t)s * 4 + 1 + a) * 512 + l] = Store<T>::ld(p + a * pstride + v);
            mask[((size_t)s * 4 + 1 + a) * 512 + l] = edge_of(m, b, l, a) ? mp : 0.0f;
        }
    }
}

// Writes a warm start into the state: u on Omega (clamped to [-1, 1]), u_bar = u, and p
// on the edges of Eq. 3, projected onto the unit ball; zero elsewhere.
template <typename T>
__global__ void apply_kernel(DeviceMap m, T* u, T* ub, T* p, size_t pstride, const int32_t* __restrict__ blocks, int n,
                             const float* __restrict__ out, int with_dual) {
    const long long total = (long long)n * kBlockVoxels;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / kBlockVoxels), l = (int)(i % kBlockVoxels);
        const int b = blocks ? blocks[s] : s;
        const int gx = (l & 7) + 1, gy = ((l >> 3) & 7) + 1, gz = (l >> 6) + 1;
        const float* o = out + ((size_t)s * kGV + gx + kG * gy + kG * kG * gz) * kC;
        const bool om = omega_of(m, b, l);
        const float u0 = om ? fminf(1.0f, fmaxf(-1.0f, o[0])) : 0.0f;
        float q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int lc = a == 0 ? (l & 7) : (a == 1 ? ((l >> 3) & 7) : (l >> 6));
            const bool keep = with_dual == 1 || (with_dual == 2 && lc < 7);  // 2: edges inside the block only
            q[a] = (keep && edge_of(m, b, l, a)) ? o[1 + a] : 0.0f;
        }
        const float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        const float sc = n2 > 1.0f ? rsqrtf(n2) : 1.0f;
        const size_t v = (size_t)b * kBlockVoxels + l;
        Store<T>::st(u + v, u0);
        Store<T>::st(ub + v, u0);
#pragma unroll
        for (int a = 0; a < 3; ++a) Store<T>::st(p + a * pstride + v, q[a] * sc);
    }
}

}  // namespace

// Divergence targets of the listed blocks from the context's state, FP32 [n][6][512]:
// 0 u, 1 Omega (1 / 0), 2 the divergence of p over the block's inner Eq. 3 edges
// (Eq. 4 with the edges that cross the block's faces left out), 3..5 the inner edge
// masks e_a(l) = Omega(l) and Omega(l + a) and l_a < 7.
template <typename T>
__global__ void targets_div_kernel(DeviceMap m, const T* u, const T* p, size_t pstride,
                                   const int32_t* __restrict__ blocks, int n, float* target) {
    const long long total = (long long)n * kBlockVoxels;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / kBlockVoxels), l = (int)(i % kBlockVoxels);
        const int b = blocks ? blocks[s] : s;
        const size_t v = (size_t)b * kBlockVoxels + l;
        const int lc[3] = {l & 7, (l >> 3) & 7, l >> 6};
        const int step[3] = {1, 8, 64};
        const bool o = omega_of(m, b, l);
        float dv = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const bool e = o && lc[a] < 7 && omega_of(m, b, l + step[a]);
            const bool eb = lc[a] > 0 && omega_of(m, b, l - step[a]) && o;
            const float own = e ? Store<T>::ld(p + a * pstride + v) : 0.0f;
            const float back = eb ? Store<T>::ld(p + a * pstride + v - step[a]) : 0.0f;
            dv = __fadd_rn(dv, __fsub_rn(own, back));
            target[((size_t)s * 6 + 3 + a) * 512 + l] = e ? 1.0f : 0.0f;
        }
        target[((size_t)s * 6 + 0) * 512 + l] = o ? Store<T>::ld(u + v) : 0.0f;
        target[((size_t)s * 6 + 1) * 512 + l] = o ? 1.0f : 0.0f;
        target[((size_t)s * 6 + 2) * 512 + l] = o ? dv : 0.0f;
    }
}

// Loss of the divergence-trained warm start, one CTA of 512 threads per sample:
//   L = (1/n) sum_samples sum_Omega [ wu (u - u*)^2 + wd (div p - div p*)^2 ]
// with u = out channel 0 and p_a = out channel 1 + a on the centre 8^3, div the inner-edge
// divergence of the targets (channel 2), and dout = dL/dout in BF16 on the 10^3 grid
// (zero off the centre and off channels 0..3).  d(div)/dp_a(l) is e_a(l) at l and -e_a(l)
// at l + a, so the p gradient is 2 wd e_a(l) (r(l) - r(l + a)) / n, r the divergence residual.
__global__ void __launch_bounds__(512) loss_div_kernel(const float* __restrict__ out, const float* __restrict__ target,
                                                       float wu, float wd, __nv_bfloat16* __restrict__ dout,
                                                       double* loss, int n) {
    __shared__ float P[3][512];
    __shared__ float R[512];
    __shared__ double red[16];
    const int s = blockIdx.x, l = threadIdx.x;
    const int lc[3] = {l & 7, (l >> 3) & 7, l >> 6};
    const int step[3] = {1, 8, 64};
    const int gv = (lc[0] + 1) + kG * (lc[1] + 1) + kG * kG * (lc[2] + 1);
    const float* o = out + ((size_t)s * kGV + gv) * kC;
    const float* tg = target + (size_t)s * 6 * 512;
    const bool om = tg[512 + l] != 0.0f;
    bool e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e[a] = tg[(3 + a) * 512 + l] != 0.0f;
        P[a][l] = e[a] ? o[1 + a] : 0.0f;
    }
    __syncthreads();
    float dv = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) dv += P[a][l] - (lc[a] > 0 ? P[a][l - step[a]] : 0.0f);
    const float rd = om ? dv - tg[2 * 512 + l] : 0.0f;
    const float ru = om ? o[0] - tg[l] : 0.0f;
    R[l] = rd;
    double acc = (double)wu * ru * ru + (double)wd * rd * rd;
    __syncthreads();
    const float inv_n = 1.0f / (float)n;
    float g[4];
    g[0] = 2.0f * wu * ru * inv_n;
#pragma unroll
    for (int a = 0; a < 3; ++a) g[1 + a] = e[a] ? 2.0f * wd * (rd - R[l + step[a]]) * inv_n : 0.0f;
    // dout: the centre voxel's four channels here, then zeros for the rest of the grid
    __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(dout + ((size_t)s * kGV + gv) * kC);
    dst[0] = __floats2bfloat162_rn(g[0], g[1]);
    dst[1] = __floats2bfloat162_rn(g[2], g[3]);
#pragma unroll
    for (int q = 2; q < kC / 2; ++q) dst[q] = __floats2bfloat162_rn(0.0f, 0.0f);
    for (int v = l; v < kGV; v += 512) {
        const int x = v % kG, y = (v / kG) % kG, z = v / (kG * kG);
        if (x >= 1 && x <= 8 && y >= 1 && y <= 8 && z >= 1 && z <= 8) continue;
        uint4* d = reinterpret_cast<uint4*>(dout + ((size_t)s * kGV + v) * kC);
        d[0] = make_uint4(0, 0, 0, 0);
        d[1] = make_uint4(0, 0, 0, 0);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((l & 31) == 0) red[l >> 5] = acc;
    __syncthreads();
    if (l == 0) {
        double t = 0.0;
        for (int i = 0; i < 16; ++i) t += red[i];
        atomicAdd(loss, t / n);
    }
}

int configure_net_kernels() {
    cudaError_t e = cudaFuncSetAttribute(conv3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kTileBytes + (size_t)kTiles * 16 * kC * 2));
    return e == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

int launch_net_targets(denser_ctx* c, const int32_t* blocks, int n, float* target, float* mask, float mu, float mp,
                       cudaStream_t s) {
    const size_t ps = (size_t)c->d.max_blocks * kBlockVoxels;
    const int g = grid_for(c->sm_count, (long long)n * kBlockVoxels, 256, 8);
    switch (c->prm.precision) {
        case DENSER_FP16:
            targets_kernel<__half><<<g, 256, 0, s>>>(c->d, (const __half*)c->d.u, (const __half*)c->d.p[c->cur], ps,
                                                     blocks, n, target, mask, mu, mp);
            break;
        case DENSER_BF16:
            targets_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(c->d, (const __nv_bfloat16*)c->d.u,
                                                            (const __nv_bfloat16*)c->d.p[c->cur], ps, blocks, n, target,
                                                            mask, mu, mp);
            break;
        default:
            targets_kernel<float><<<g, 256, 0, s>>>(c->d, (const float*)c->d.u, (const float*)c->d.p[c->cur], ps,
                                                    blocks, n, target, mask, mu, mp);
    }
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "targets kernel");
}

int launch_net_targets_div(denser_ctx* c, const int32_t* blocks, int n, float* target, cudaStream_t s) {
    const size_t ps = (size_t)c->d.max_blocks * kBlockVoxels;
    const int g = grid_for(c->sm_count, (long long)n * kBlockVoxels, 256, 8);
    switch (c->prm.precision) {
        case DENSER_FP16:
            targets_div_kernel<__half><<<g, 256, 0, s>>>(c->d, (const __half*)c->d.u, (const __half*)c->d.p[c->cur],
                                                         ps, blocks, n, target);
            break;
        case DENSER_BF16:
            targets_div_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(c->d, (const __nv_bfloat16*)c->d.u,
                                                                (const __nv_bfloat16*)c->d.p[c->cur], ps, blocks, n,
                                                                target);
            break;
        default:
            targets_div_kernel<float><<<g, 256, 0, s>>>(c->d, (const float*)c->d.u, (const float*)c->d.p[c->cur], ps,
                                                        blocks, n, target);
    }
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "divergence targets kernel");
}

int launch_net_apply(denser_ctx* c, const int32_t* blocks, int n, const float* out, int with_dual, cudaStream_t s) {
    const size_t ps = (size_t)c->d.max_blocks * kBlockVoxels;
    const int g = grid_for(c->sm_count, (long long)n * kBlockVoxels, 256, 8);
    const int cur = c->cur;
    switch (c->prm.precision) {
        case DENSER_FP16:
            apply_kernel<__half><<<g, 256, 0, s>>>(c->d, (__half*)c->d.u, (__half*)c->d.ub[cur], (__half*)c->d.p[cur], ps,
                                                   blocks, n, out, with_dual);
            break;
        case DENSER_BF16:
            apply_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(c->d, (__nv_bfloat16*)c->d.u, (__nv_bfloat16*)c->d.ub[cur],
                                                          (__nv_bfloat16*)c->d.p[cur], ps, blocks, n, out, with_dual);
            break;
        default:
            apply_kernel<float><<<g, 256, 0, s>>>(c->d, (float*)c->d.u, (float*)c->d.ub[cur], (float*)c->d.p[cur], ps,
                                                  blocks, n, out, with_dual);
    }
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "apply kernel");
}

int launch_net_gather(denser_ctx* c, const int32_t* blocks, int n, void* x, cudaStream_t s) {
    gather_kernel<<<std::min(n, c->sm_count * 8), 256, 0, s>>>(c->d, blocks, n, (__nv_bfloat16*)x);
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "gather kernel");
}

}  // namespace denser

// ------------------------------------------------------------- context-free calls
using namespace denser;

static int net_grid(int n, int per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    return std::max(1, std::min(n, sms * per_sm));
}

static int net_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

extern "C" int denser_conv3(const void* x, const void* w, const float* bias, int32_t relu, void* y_bf16, float* y_f32,
                            int64_t n, void* stream) {
    if (!x || !w || n < 0 || (!y_bf16 && !y_f32)) return DENSER_ERR_INVALID_ARG;
    if (n == 0) return DENSER_OK;
    if (configure_net_kernels() != DENSER_OK) return DENSER_ERR_CUDA;
    conv3_tc_kernel<<<net_grid((int)n, 2), kNetThreads, kTcSmem, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)x, (const __nv_bfloat16*)w, bias, relu, (__nv_bfloat16*)y_bf16, y_f32, (int)n);
    return net_status();
}

extern "C" int denser_net_check(void* stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return DENSER_ERR_CUDA;
    }
    int lost = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&lost, g_tc_timeout, sizeof(int)) != cudaSuccess ||
        (lost && cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int)) != cudaSuccess)) {
        cudaGetLastError();
        return DENSER_ERR_CUDA;
    }
    return lost ? DENSER_ERR_TIMEOUT : DENSER_OK;
}

extern "C" int denser_conv3_wgrad(const void* h, const void* dz, float* dw, float* db, int64_t n, void* stream) {
    if (!h || !dz || !dw || !db || n < 0) return DENSER_ERR_INVALID_ARG;
    if (n == 0) return DENSER_OK;
    if (configure_net_kernels() != DENSER_OK) return DENSER_ERR_CUDA;
    wgrad_kernel<<<net_grid((int)n, 2), kNetThreads, kTileBytes + (size_t)kTiles * 16 * kC * 2, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)h, (const __nv_bfloat16*)dz, dw, db, (int)n);
    return net_status();
}

extern "C" int denser_relu_backward(const void* dh, const void* h, void* dz, int64_t count, void* stream) {
    if (!dh || !h || !dz || count < 0) return DENSER_ERR_INVALID_ARG;
    if (count == 0) return DENSER_OK;
    relu_backward_kernel<<<net_grid((int)std::min<int64_t>(count / 256 + 1, 1 << 20), 16), 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)dh, (const __nv_bfloat16*)h, (__nv_bfloat16*)dz, count);
    return net_status();
}

extern "C" int denser_net_loss(const float* out, const float* target, const float* mask, void* dout, double* loss,
                               int64_t n, void* stream) {
    if (!out || !target || !mask || !dout || !loss || n <= 0) return DENSER_ERR_INVALID_ARG;
    loss_kernel<<<net_grid((int)std::min<int64_t>(n * kGV / 256 + 1, 1 << 20), 8), 256, 0, (cudaStream_t)stream>>>(
        out, target, mask, (__nv_bfloat16*)dout, loss, (int)n);
    return net_status();
}

extern "C" int denser_net_loss_div(const float* out, const float* target, float u_weight, float div_weight,
                                   void* dout, double* loss, int64_t n, void* stream) {
    if (!out || !target || !dout || !loss || n <= 0 || n > (1 << 30) || !(u_weight >= 0) || !(div_weight >= 0))
        return DENSER_ERR_INVALID_ARG;
    loss_div_kernel<<<(unsigned)n, 512, 0, (cudaStream_t)stream>>>(out, target, u_weight, div_weight,
                                                                   (__nv_bfloat16*)dout, loss, (int)n);
    return net_status();
}

extern "C" int denser_adam(float* w, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                           float beta2, float eps, int32_t step, void* stream) {
    if (!w || !grad || !m || !v || count < 0 || step < 1) return DENSER_ERR_INVALID_ARG;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    adam_kernel<<<net_grid((int)(count / 256 + 1), 4), 256, 0, (cudaStream_t)stream>>>(w, grad, m, v, (int)count, lr, beta1,
                                                                                       beta2, eps, c1, c2);
    return net_status();
}

extern "C" int denser_pack_weights(const float* w32, void* wf, void* wb, void* stream) {
    if (!w32 || !wf || !wb) return DENSER_ERR_INVALID_ARG;
    pack_weights_kernel<<<16, 256, 0, (cudaStream_t)stream>>>(w32, (__nv_bfloat16*)wf, (__nv_bfloat16*)wb);
    return net_status();
}
