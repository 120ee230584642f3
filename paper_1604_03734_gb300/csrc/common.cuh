// Internal declarations shared by the DENSER CUDA translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/denser.h"

namespace denser {

constexpr int kBlock = 8;
constexpr int kBlockVoxels = 512;
constexpr int kNeighbours = 12;
constexpr int kVisOriginFloats = 12;      // words per (listed block, map) entry of the fusion origins
constexpr int kMaxProbe = 512;             // linear-probe limit of the hash table
constexpr int kSortChunk = 2048;           // keys sorted per CTA before the rank merge (block order)
constexpr int kNewKeyChunk = 512;          // the same for an allocation call's new keys (a few thousand:
                                           // several CTAs sort at once)
constexpr int kSweepThreads = 512;
constexpr int kInvWeights = 4096;          // integer counts w whose 1/(2 lambda w) the energy reads from a table
// Largest block pool a context accepts.  Voxel offsets (block * 512 + l) are computed in
// 64 bits everywhere; block indices are 32-bit, and 2^24 blocks (8.6 G voxels, about
// 400 GB of FP32 state) is beyond any one device's memory.
constexpr uint32_t kMaxPoolBlocks = 1u << 24;
constexpr int kMaxBatch = 16;              // depth maps per batched allocation + fusion launch

// ---------------------------------------------------------------- block keys
// 64-bit key: bits 0-18 bx + 2^18, 19-37 by + 2^18, 38-56 bz + 2^18, 57-63 segment.
// Ascending keys = ascending (segment, bz, by, bx).  Segment 127 is reserved, so the
// all-ones word never is a key and marks an empty hash slot.
constexpr int kCoordBits = 19;
constexpr int32_t kCoordBias = 1 << 18;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int32_t kMaxSegment = 126;

__host__ __device__ inline bool key_in_range(int32_t seg, long long bx, long long by, long long bz) {
    return seg >= 0 && seg <= kMaxSegment && bx >= -kCoordBias && bx < kCoordBias &&
           by >= -kCoordBias && by < kCoordBias && bz >= -kCoordBias && bz < kCoordBias;
}

__host__ __device__ inline unsigned long long pack_key(int32_t seg, int32_t bx, int32_t by, int32_t bz) {
    return (unsigned long long)(uint32_t)(bx + kCoordBias) |
           ((unsigned long long)(uint32_t)(by + kCoordBias) << kCoordBits) |
           ((unsigned long long)(uint32_t)(bz + kCoordBias) << (2 * kCoordBits)) |
           ((unsigned long long)(uint32_t)seg << (3 * kCoordBits));
}

__host__ __device__ inline void unpack_key(unsigned long long k, int32_t* seg, int32_t* bx, int32_t* by,
                                           int32_t* bz) {
    const unsigned long long m = (1ull << kCoordBits) - 1;
    *bx = (int32_t)(k & m) - kCoordBias;
    *by = (int32_t)((k >> kCoordBits) & m) - kCoordBias;
    *bz = (int32_t)((k >> (2 * kCoordBits)) & m) - kCoordBias;
    *seg = (int32_t)(k >> (3 * kCoordBits));
}

// Spatial hash of Teschner et al. (large primes XORed), plus the segment.
__host__ __device__ inline uint32_t hash_key(unsigned long long k) {
    int32_t s, x, y, z;
    unpack_key(k, &s, &x, &y, &z);
    return ((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349669u) ^ ((uint32_t)z * 83492791u) ^
           ((uint32_t)s * 2654435761u);
}

// The hardware's approximate reciprocal: at most 1 ulp from 1/x for normal x (denormal
// inputs and results are flushed to zero, which no caller produces).
__device__ inline float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;\n" : "=f"(r) : "f"(x));
    return r;
}

// --------------------------------------------------------- device-side words
enum Counter {
    kNumBlocks = 0,    // allocated blocks
    kNumNew = 1,       // keys inserted by the running allocation call
    kLastNew = 2,      // blocks added by the last allocation call
    kErrorBits = 3,    // sticky error flags (ErrorBit)
    kNumVisible = 4,   // blocks selected for the running fusion call
    kNumCounters = 8,  // words copied to the host
    kFrameDepthMax = 8,  // [kMaxBatch] max valid depth per depth map of the running call (float bits)
    kCounterWords = kFrameDepthMax + kMaxBatch
};

enum ErrorBit : int32_t {
    kErrHashFull = 1,
    kErrPoolFull = 2,
    kErrNewFull = 4,
    kErrRange = 8,
    kErrTimeout = 16,
    kErrDuplicate = 32,
};

// Storage of the primal-dual fields.
template <typename T> struct Store;
template <> struct Store<float> {
    __device__ static float ld(const float* p) { return *p; }
    __device__ static void st(float* p, float v) { *p = v; }
};
// The 16-bit types also convert pairs (a 32-bit word, lower address in the low half):
// the same values as two single conversions, in fewer instructions.
template <> struct Store<__half> {
    __device__ static float ld(const __half* p) { return __half2float(*p); }
    __device__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
    __device__ static float2 ld2(uint32_t w) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    __device__ static uint32_t st2(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <> struct Store<__nv_bfloat16> {
    __device__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static float2 ld2(uint32_t w) {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        return __bfloat1622float2(h);
    }
    __device__ static uint32_t st2(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

// All device pointers of one context.
struct DeviceMap {
    unsigned long long* hash_keys;  // [slots]
    int32_t* hash_vals;             // [slots] block index; -1 pending, -2 rejected
    int32_t* hash_birth;            // [slots] first depth map of the running batch that
                                    // reached the slot's key (atomic min; 0x7f7f7f7f: none)
    uint8_t* block_birth;           // [max_blocks] that depth map, for the blocks a batch added
    uint32_t slot_mask;
    int32_t* coords;                // [max_blocks][4] (segment, bx, by, bz)
    float* f;                       // [max_blocks][512]
    float* w;                       // [max_blocks][512]
    void* u;                        // [max_blocks][512] storage type
    void* ub[2];                    // ping-pong u_bar
    void* p[2];                     // ping-pong p, [3][max_blocks][512]
    uint32_t* omega_bits;           // [max_blocks][16]
    int32_t* nbr;                   // [max_blocks][12]
    int32_t* counters;              // [kNumCounters]
    unsigned long long* new_keys;   // [max_new] inserted keys of the running call
    uint32_t* new_slots;            // [max_new]
    int32_t* visible;               // [max_blocks] fusion work list ({block, depth-map mask})
    float* vis_org;                 // [max_blocks][org_frames][kVisOriginFloats] the listed blocks'
                                    // camera-frame origins per depth map (float32 hi, lo, bound)
                                    // and their voxels' shared projection bounds
    int32_t org_frames;             // depth maps per entry that vis_org holds
    double* partials;               // [kEnergyGrid][2] energy partial sums
    uint32_t max_blocks;
    uint32_t max_new;
};

constexpr int kEnergyGrid = 1216;  // 8 CTAs per SM on 152 SMs

}  // namespace denser

// ------------------------------------------------------------------ the context
struct denser_ctx {
    denser_params prm;
    int device;
    int sm_count;
    denser::DeviceMap d;
    size_t elem_size;          // bytes per stored u / u_bar / p element
    int cur;                   // which ping-pong buffer holds the current u_bar and p
    int64_t nbr_valid_blocks;  // blocks covered by the neighbour table (-1: rebuild)
    float* stage;              // device staging for host inputs
    size_t stage_bytes;
    // depth maps from host memory: two device buffers filled on copy_stream, so that a
    // frame's copy overlaps the previous frame's kernels
    cudaStream_t copy_stream;
    float* dstage[2];
    size_t dstage_bytes[2];
    cudaEvent_t dstage_copied[2];  // recorded on copy_stream after the copy into dstage[i]
    cudaEvent_t dstage_free[2];    // recorded on the call's stream after the kernels reading dstage[i]
    int dstage_next;
    // laser fusion: per-voxel packed accumulators (count << 48 plus a fixed-point sum)
    // and per-block touched flags, allocated on first use
    unsigned long long* laser_acc;
    uint8_t* laser_touched;
    void* hstage;              // pinned host staging for host outputs
    size_t hstage_bytes;
    uint8_t* omega_bytes;      // extract scratch
    float* conv_scratch;       // float32 staging of converted state
    size_t conv_bytes;
    int32_t* surf_counts;      // [max_blocks] triangles per block (surface extraction)
    long long* surf_offsets;   // [max_blocks + 1] their exclusive scan
    int32_t* surf_up;          // [max_blocks][8] upper-neighbour block indices
    unsigned long long* surf_list;    // cubes with triangles (count pass)
    long long surf_list_cap;
    unsigned long long* surf_cursor;  // device: entries the count pass produced
    long long surf_items;             // host copy of *surf_cursor
    void* surf_scratch;        // device staging of host surface outputs
    size_t surf_bytes;
    int32_t* h_counters;       // pinned copy of the device counters
    double* h_energy;          // pinned [2]
    unsigned long long launches;
    denser_schedule sched;     // sweep schedule
    int32_t* order;            // [max_blocks] sweep visiting order (sorted keys)
    unsigned long long* order_keys;  // [max_blocks] scratch of the order sort
    uint32_t* order_vals;      // [max_blocks]
    int64_t order_valid_blocks;  // blocks covered by `order` (-1: rebuild)
    // graph-captured iteration loop (schedule.use_graph)
    cudaStream_t capture_stream;   // private stream used only to record graphs
    int32_t* ctl_i;                // device [4]: iterations done, max iterations, converged, gap evaluations
    double* ctl_d;                 // device [4]: gap tolerance, P, D, unused
    int32_t* h_ctl_i;              // pinned copies
    double* h_ctl_d;
    struct LoopGraph {
        bool valid;
        int64_t nb;
        denser_schedule sched;
        int cur, k, with_gap;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
    } loop;
    // fusion profiling (denser_set_fusion_profiling): events recorded before the key
    // pass, after it, after the rest of the allocation, after culling and origins, and
    // after the fusion kernel of each batched group
    bool profile;
    cudaEvent_t prof_ev[5];
    denser_fusion_profile prof;
    std::string msg;
};

namespace denser {

// Launchers implemented in the .cu files (all enqueue on `s`).
// Allocation for n_frames (1..kMaxBatch) depth maps of one camera, stored back to back
// ([n_frames][H][W] float32), with poses T [n_frames][16]: one key pass over all of
// them, then one sort / index / zero / commit.  New blocks are indexed in order of
// (first depth map that reached them, key), the order that one call per depth map
// gives.  The pass also records each map's largest valid depth and resets the fusion's
// visible count.
int launch_alloc(denser_ctx* c, const float* depth_dev, int n_frames, const denser_intrinsics* K, const double* T,
                 int32_t segment, cudaStream_t s);
// Fusion of the same n_frames depth maps: one culling pass and one fusion pass, each
// voxel taking the maps in order.  after_alloc: launch_alloc of the same maps ran just
// before (their depth maxima are recorded, and a block that the batch added is fused
// only from the first map that allocated it on, as one call per map would); otherwise
// the depth maxima are computed here and every allocated block takes every map.
int launch_fuse(denser_ctx* c, const float* depth_dev, int n_frames, const denser_intrinsics* K, const double* T,
                int32_t segment, cudaStream_t s, bool after_alloc = false);
int launch_load_blocks(denser_ctx* c, const int32_t* coords_dev, int64_t n, int64_t base, cudaStream_t s);
int launch_prepare_regularize(denser_ctx* c, int64_t n_blocks, bool rebuild_nbr, cudaStream_t s);
int launch_sweep(denser_ctx* c, int64_t n_blocks, cudaStream_t s);
int launch_energy(denser_ctx* c, int64_t n_blocks, cudaStream_t s);
int launch_omega_bytes(denser_ctx* c, int64_t n_blocks, uint8_t* out, cudaStream_t s);
int launch_convert_state(denser_ctx* c, const void* src, float* dst, int64_t n, bool to_float,
                         cudaStream_t s);
int launch_surface(denser_ctx* c, int64_t nb, int pass, float* tri_pos, long long* tri_ids, int64_t capacity,
                   cudaStream_t s);
int launch_alloc_points(denser_ctx* c, const float* pts, int64_t n, const double* T, int32_t segment, cudaStream_t s);
int stereo_census(const float* img, int W, int H, unsigned long long* sig, cudaStream_t s);
int stereo_tensor(const float* img, int W, int H, float gamma, float beta, float* T, cudaStream_t s);
int stereo_assign(const unsigned long long* sigL, const unsigned long long* sigR, int W, int H, int D, float lambda,
                  double theta, const float* d, float* a, cudaStream_t s);
int stereo_tgv(const float* a, const float* T, int W, int H, float alpha1, float alpha2, double theta, int iters,
               float* state, cudaStream_t s);
int stereo_init_state(float* state, const float* d0, int W, int H, cudaStream_t s);
int stereo_depth(const float* disp, int W, int H, float fb, float min_disp, float* depth, cudaStream_t s);
int launch_fuse_points(denser_ctx* c, const float* pts, int64_t n, const double* T, int32_t segment, cudaStream_t s);
int launch_zero_state(denser_ctx* c, int64_t first_block, int64_t n_blocks, cudaStream_t s);
int launch_block_order(denser_ctx* c, int64_t n_blocks, cudaStream_t s);
int configure_kernels(denser_ctx* c);
int launch_graph_loop(denser_ctx* c, int64_t n_blocks, int k, bool with_gap, cudaStream_t s);
int launch_net_gather(denser_ctx* c, const int32_t* blocks, int n, void* x, cudaStream_t s);
int launch_net_targets_div(denser_ctx* c, const int32_t* blocks, int n, float* target, cudaStream_t s);
int launch_net_targets(denser_ctx* c, const int32_t* blocks, int n, float* target, float* mask, float mu, float mp,
                       cudaStream_t s);
int launch_net_apply(denser_ctx* c, const int32_t* blocks, int n, const float* out, int with_dual, cudaStream_t s);
void release_graph_loop(denser_ctx* c);

int set_error(denser_ctx* c, int code, const std::string& m);
int cuda_check(denser_ctx* c, cudaError_t e, const char* what);

}  // namespace denser

namespace denser {

// Lookup of a block key; returns the block index or -1 (absent, pending or rejected).
__device__ inline int32_t hash_lookup(const DeviceMap& m, unsigned long long key) {
    const uint32_t h = hash_key(key);
    for (int i = 0; i < kMaxProbe; ++i) {
        const uint32_t slot = (h + (uint32_t)i) & m.slot_mask;
        const unsigned long long k = __ldcg(m.hash_keys + slot);
        if (k == key) return __ldcg(m.hash_vals + slot);
        if (k == kEmptyKey) return -1;
    }
    return -1;
}

// Neighbour slots of the 12-entry table: 6 faces, then the 6 (low, high) edges that
// the fused primal-dual sweep reads.
__host__ __device__ inline void neighbour_offset(int i, int* dx, int* dy, int* dz) {
    const signed char t[kNeighbours][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {-1, 0, 0},
                                           {0, -1, 0}, {0, 0, -1}, {-1, 1, 0}, {-1, 0, 1},
                                           {1, -1, 0}, {0, -1, 1}, {1, 0, -1}, {0, 1, -1}};
    *dx = t[i][0];
    *dy = t[i][1];
    *dz = t[i][2];
}

// floor(v) for |v| < 2^22 with plain round-to-nearest FP32 arithmetic and integer
// operations: v + 1.5*2^23 lands in [2^23, 2^24), where the float spacing is 1, so it
// rounds to n + 1.5*2^23 with n the integer nearest v, held in its mantissa; floor(v)
// is n, or n - 1 when n > v.  (Conversions from float to 64-bit integers, rounding
// instructions and directed-rounding adds are avoided: this GPU runs some of them on
// its narrow FP64 pipe.)
__device__ inline int floor_small(float v) {
    const float t = __fadd_rn(v, 12582912.0f);
    const int n = __float_as_int(t) - 0x4B400000;
    return (t - 12582912.0f) > v ? n - 1 : n;
}

// Ray of a laser point p (sensor frame) under a sensor->global rotation R (row-major):
// range r = sqrt((x*x + y*y) + z*z), unit direction d = p / r and its global direction
// dg = R d, each row summed left to right, every float64 operation rounded on its own
// (the _rn intrinsics keep fused multiply-adds out).  Returns false for a point that is
// not finite or at range 0.
__device__ inline bool laser_ray(const double* R, float px, float py, float pz, double* r, double* dg) {
    const double x = px, y = py, z = pz;
    const double rr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    if (!(isfinite(rr) && rr > 0.0)) return false;
    const double d0 = __ddiv_rn(x, rr), d1 = __ddiv_rn(y, rr), d2 = __ddiv_rn(z, rr);
#pragma unroll
    for (int i = 0; i < 3; ++i)
        dg[i] = __dadd_rn(__dadd_rn(__dmul_rn(R[3 * i], d0), __dmul_rn(R[3 * i + 1], d1)), __dmul_rn(R[3 * i + 2], d2));
    *r = rr;
    return true;
}

inline int grid_for(int sm_count, long long work, int threads, int per_sm) {
    long long g = (work + threads - 1) / threads;
    long long cap = (long long)sm_count * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace denser
