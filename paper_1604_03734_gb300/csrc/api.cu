// C ABI of the DENSER hot path: context, argument checks, host/device staging,
// the regularisation loop and the copies out.  The kernels live in alloc.cu,
// fuse.cu and regularize.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>
#include <string>

#include <initializer_list>

#include "common.cuh"

using namespace denser;

namespace denser {

int set_error(denser_ctx* c, int code, const std::string& m) {
    if (c) c->msg = m;
    return code;
}

int cuda_check(denser_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return DENSER_OK;
    return set_error(c, DENSER_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace denser

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure_stage(denser_ctx* c, size_t bytes) {
    if (c->stage_bytes >= bytes) return DENSER_OK;
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    int rc = cuda_check(c, cudaMalloc(&c->stage, bytes), "cudaMalloc(stage)");
    if (rc) return rc;
    c->stage_bytes = bytes;
    return DENSER_OK;
}

int ensure_conv(denser_ctx* c, size_t bytes) {
    if (c->conv_bytes >= bytes) return DENSER_OK;
    if (c->conv_scratch) cudaFree(c->conv_scratch);
    c->conv_scratch = nullptr;
    c->conv_bytes = 0;
    int rc = cuda_check(c, cudaMalloc(&c->conv_scratch, bytes), "cudaMalloc(convert scratch)");
    if (rc) return rc;
    c->conv_bytes = bytes;
    return DENSER_OK;
}

// Returns a device pointer holding `bytes` of `src`: src itself when it is device
// memory, else a copy in the context's staging buffer.
int device_input(denser_ctx* c, const void* src, size_t bytes, cudaStream_t s, const void** out) {
    if (is_device_ptr(src)) {
        *out = src;
        return DENSER_OK;
    }
    int rc = ensure_stage(c, bytes);
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpyAsync(c->stage, src, bytes, cudaMemcpyDefault, s), "copy input to device");
    if (rc) return rc;
    *out = c->stage;
    return DENSER_OK;
}

// A device pointer to a depth map: `src` itself when it is device memory, else a copy
// made on the context's copy stream into the next of two staging buffers.  The copy
// waits until the kernels that read that buffer two frames ago are done, and `s` waits
// for the copy; *slot names the buffer for release_depth (-1: none).
int stage_depth(denser_ctx* c, const float* src, size_t bytes, cudaStream_t s, const float** out, int* slot) {
    *slot = -1;
    if (is_device_ptr(src)) {
        *out = src;
        return DENSER_OK;
    }
    const int i = c->dstage_next;
    c->dstage_next ^= 1;
    int rc;
    if (c->dstage_bytes[i] < bytes) {
        // the buffer may still be read by queued kernels: wait for them before freeing
        if (c->dstage[i]) {
            if ((rc = cuda_check(c, cudaEventSynchronize(c->dstage_free[i]), "wait for staging buffer"))) return rc;
            cudaFree(c->dstage[i]);
        }
        c->dstage[i] = nullptr;
        c->dstage_bytes[i] = 0;
        if ((rc = cuda_check(c, cudaMalloc(&c->dstage[i], bytes), "cudaMalloc(depth staging)"))) return rc;
        c->dstage_bytes[i] = bytes;
    }
    if ((rc = cuda_check(c, cudaStreamWaitEvent(c->copy_stream, c->dstage_free[i], 0), "copy stream wait"))) return rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(c->dstage[i], src, bytes, cudaMemcpyHostToDevice, c->copy_stream),
                         "copy depth to device")))
        return rc;
    if ((rc = cuda_check(c, cudaEventRecord(c->dstage_copied[i], c->copy_stream), "record copy"))) return rc;
    if ((rc = cuda_check(c, cudaStreamWaitEvent(s, c->dstage_copied[i], 0), "stream wait for copy"))) return rc;
    *out = c->dstage[i];
    *slot = i;
    return DENSER_OK;
}

// Marks staging buffer `slot` free once the work queued so far on `s` is done.
int release_depth(denser_ctx* c, int slot, cudaStream_t s) {
    if (slot < 0) return DENSER_OK;
    return cuda_check(c, cudaEventRecord(c->dstage_free[slot], s), "record staging release");
}

int device_error_code(denser_ctx* c, int32_t bits) {
    if (!bits) return DENSER_OK;
    if (bits & kErrHashFull) return set_error(c, DENSER_ERR_HASH_FULL, "hash table full (probe limit reached)");
    if (bits & (kErrPoolFull | kErrNewFull))
        return set_error(c, DENSER_ERR_POOL_FULL, "block pool or per-call new-block capacity exhausted");
    if (bits & kErrRange) return set_error(c, DENSER_ERR_RANGE, "block coordinate out of range (|b| >= 2^18)");
    if (bits & kErrTimeout) return set_error(c, DENSER_ERR_TIMEOUT, "device-side wait gave up");
    if (bits & kErrDuplicate) return set_error(c, DENSER_ERR_INVALID_ARG, "block already present in the map");
    return set_error(c, DENSER_ERR_CUDA, "unknown device error bits");
}

// Waits for the stream and refreshes the host copy of the counters.
int read_counters(denser_ctx* c, cudaStream_t s) {
    int rc = cuda_check(c, cudaMemcpyAsync(c->h_counters, c->d.counters, kNumCounters * sizeof(int32_t),
                                           cudaMemcpyDeviceToHost, s),
                        "read counters");
    if (rc) return rc;
    rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
    if (rc) return rc;
    return device_error_code(c, c->h_counters[kErrorBits]);
}

bool valid_intrinsics(const denser_intrinsics* K) {
    return K && K->width > 0 && K->height > 0 && K->width <= (1 << 20) && K->height <= (1 << 20) &&
           (int64_t)K->width * K->height < (1ll << 31) &&
           isfinite(K->fx) && isfinite(K->fy) && isfinite(K->cx) && isfinite(K->cy) && K->fx > 0 && K->fy > 0;
}

bool valid_pose(const double* T) {
    if (!T) return false;
    for (int i = 0; i < 16; ++i)
        if (!isfinite(T[i])) return false;
    return T[12] == 0.0 && T[13] == 0.0 && T[14] == 0.0 && T[15] == 1.0;
}

template <typename F>
int guarded(denser_ctx* c, F&& fn) {
    if (!c) return DENSER_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    c->msg.clear();
    return fn();
}

int copy_out(denser_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t s, const char* what) {
    return cuda_check(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s), what);
}

// Copies a stored-precision field out as float32.
int copy_state_out(denser_ctx* c, float* dst, const void* src, int64_t n, cudaStream_t s) {
    if (c->prm.precision == DENSER_FP32) return copy_out(c, dst, src, (size_t)n * 4, s, "copy state out");
    int rc = ensure_conv(c, (size_t)n * 4);
    if (rc) return rc;
    rc = launch_convert_state(c, src, c->conv_scratch, n, true, s);
    if (rc) return rc;
    return copy_out(c, dst, c->conv_scratch, (size_t)n * 4, s, "copy state out");
}

int copy_state_in(denser_ctx* c, void* dst, const float* src, int64_t n, cudaStream_t s) {
    if (!src) return cuda_check(c, cudaMemsetAsync(dst, 0, (size_t)n * c->elem_size, s), "zero state");
    if (c->prm.precision == DENSER_FP32) return copy_out(c, dst, src, (size_t)n * 4, s, "copy state in");
    int rc = ensure_conv(c, (size_t)n * 4);
    if (rc) return rc;
    rc = copy_out(c, c->conv_scratch, src, (size_t)n * 4, s, "copy state in");
    if (rc) return rc;
    return launch_convert_state(c, c->conv_scratch, (float*)dst, n, false, s);
}

int energy_now(denser_ctx* c, int64_t nb, cudaStream_t s, double* P, double* D) {
    int rc = launch_energy(c, nb, s);
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpyAsync(c->h_energy, c->d.partials + 2 * kEnergyGrid, 2 * sizeof(double),
                                       cudaMemcpyDeviceToHost, s),
                    "read energies");
    if (rc) return rc;
    rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
    if (rc) return rc;
    *P = c->h_energy[0];
    *D = c->h_energy[1];
    return DENSER_OK;
}

void free_all(denser_ctx* c) {
    void* ptrs[] = {c->d.hash_keys, c->d.hash_vals, c->d.hash_birth, c->d.block_birth, c->d.coords, c->d.f, c->d.w, c->d.u, c->d.ub[0], c->d.ub[1],
                    c->d.p[0], c->d.p[1], c->d.omega_bits, c->d.nbr, c->d.counters, c->d.new_keys,
                    c->d.new_slots, c->d.visible, c->d.vis_org, c->d.partials, c->stage, c->omega_bytes, c->conv_scratch,
                    c->order, c->order_keys, c->order_vals, c->ctl_i, c->ctl_d, c->surf_counts,
                    c->surf_offsets, c->surf_scratch, c->surf_up, c->surf_list, c->surf_cursor};
    release_graph_loop(c);
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_counters) cudaFreeHost(c->h_counters);
    if (c->h_energy) cudaFreeHost(c->h_energy);
    if (c->h_ctl_i) cudaFreeHost(c->h_ctl_i);
    if (c->h_ctl_d) cudaFreeHost(c->h_ctl_d);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    for (int i = 0; i < 2; ++i) {
        if (c->dstage[i]) cudaFree(c->dstage[i]);
        if (c->dstage_copied[i]) cudaEventDestroy(c->dstage_copied[i]);
        if (c->dstage_free[i]) cudaEventDestroy(c->dstage_free[i]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->laser_acc) cudaFree(c->laser_acc);
    if (c->laser_touched) cudaFree(c->laser_touched);
    for (cudaEvent_t e : c->prof_ev)
        if (e) cudaEventDestroy(e);
}

}  // namespace

extern "C" {

void denser_default_params(denser_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->voxel_size = 0.1;
    p->mu = 0.3;
    p->lambda = 0.8;
    p->sigma = 0.5;
    p->tau = 1.0 / 6.0;
    p->theta = 1.0;
    p->hash_slots = 1u << 20;
    p->max_blocks = 65536;
    p->max_new_blocks = 0;
    p->precision = DENSER_FP32;
    p->gap_every = 0;
}

int denser_create(const denser_params* prm, int32_t device, denser_ctx** out) {
    if (!prm || !out) return DENSER_ERR_INVALID_ARG;
    *out = nullptr;
    const denser_params& p = *prm;
    if (!(p.voxel_size > 0) || !(p.mu > 0) || !(p.lambda > 0) || !(p.sigma > 0) || !(p.tau > 0) ||
        !(p.theta >= 0) || !isfinite(p.voxel_size) || !isfinite(p.mu) || p.max_blocks == 0 ||
        p.max_blocks > kMaxPoolBlocks || p.hash_slots < 2 || (p.hash_slots & (p.hash_slots - 1)) ||
        p.hash_slots <= p.max_blocks || p.precision < DENSER_FP32 || p.precision > DENSER_BF16 || p.gap_every < 0)
        return DENSER_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DENSER_ERR_CUDA;
    }
    denser_ctx* c = new denser_ctx();
    memset(&c->d, 0, sizeof(c->d));
    c->prm = p;
    c->device = device;
    c->cur = 0;
    c->nbr_valid_blocks = -1;
    c->stage = nullptr, c->stage_bytes = 0, c->hstage = nullptr, c->hstage_bytes = 0;
    c->omega_bytes = nullptr, c->conv_scratch = nullptr, c->conv_bytes = 0;
    c->surf_counts = nullptr, c->surf_offsets = nullptr, c->surf_scratch = nullptr, c->surf_bytes = 0;
    c->surf_up = nullptr, c->surf_list = nullptr, c->surf_list_cap = 0, c->surf_cursor = nullptr;
    c->surf_items = 0;
    c->h_counters = nullptr, c->h_energy = nullptr;
    c->launches = 0;
    // the row sweep with balanced face items and asynchronous halos, 10 CTAs per SM,
    // blocks in index order: the autotuner's pick for every storage type on the 1 km
    // street (for 16-bit storage, halos through registers are 2% faster on the 100 m
    // street but 12-17% slower on the 1 km one)
    c->sched.sweep_kernel = 7;
    c->sched.order = 0;
    c->sched.ctas_per_sm = 2;
    c->sched.use_graph = 1;
    c->order = nullptr, c->order_keys = nullptr, c->order_vals = nullptr;
    c->order_valid_blocks = -1;
    c->capture_stream = nullptr;
    c->copy_stream = nullptr;
    for (int i = 0; i < 2; ++i) {
        c->dstage[i] = nullptr, c->dstage_bytes[i] = 0;
        c->dstage_copied[i] = nullptr, c->dstage_free[i] = nullptr;
    }
    c->dstage_next = 0;
    c->laser_acc = nullptr, c->laser_touched = nullptr;
    c->ctl_i = nullptr, c->ctl_d = nullptr, c->h_ctl_i = nullptr, c->h_ctl_d = nullptr;
    c->loop.valid = false;
    c->elem_size = p.precision == DENSER_FP32 ? 4 : 2;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    const size_t mb = p.max_blocks;
    const size_t nv = mb * kBlockVoxels;
    const size_t max_new = p.max_new_blocks ? std::min<size_t>(p.max_new_blocks, mb) : mb;
    c->d.max_blocks = (uint32_t)mb;
    c->d.max_new = (uint32_t)max_new;
    c->d.slot_mask = p.hash_slots - 1;
    c->d.org_frames = 1;  // grown to kMaxBatch by the first batched fusion
    struct Req {
        void** ptr;
        size_t bytes;
    } reqs[] = {{(void**)&c->d.hash_keys, (size_t)p.hash_slots * 8},
                {(void**)&c->d.hash_vals, (size_t)p.hash_slots * 4},
                {(void**)&c->d.hash_birth, (size_t)p.hash_slots * 4},
                {(void**)&c->d.block_birth, mb},
                {(void**)&c->d.coords, mb * 16},
                {(void**)&c->d.f, nv * 4},
                {(void**)&c->d.w, nv * 4},
                {(void**)&c->d.u, nv * c->elem_size},
                {(void**)&c->d.ub[0], nv * c->elem_size},
                {(void**)&c->d.ub[1], nv * c->elem_size},
                {(void**)&c->d.p[0], 3 * nv * c->elem_size},
                {(void**)&c->d.p[1], 3 * nv * c->elem_size},
                {(void**)&c->d.omega_bits, mb * 64},
                {(void**)&c->d.nbr, mb * kNeighbours * 4},
                {(void**)&c->d.counters, kCounterWords * 4},
                {(void**)&c->d.new_keys, max_new * 8},
                {(void**)&c->d.new_slots, max_new * 4},
                {(void**)&c->d.visible, mb * 32},
                {(void**)&c->d.vis_org, mb * 4 * kVisOriginFloats},
                {(void**)&c->d.partials, (2 * (size_t)kEnergyGrid + 2 + kInvWeights) * 8},
                {(void**)&c->order, mb * 4},
                {(void**)&c->order_keys, mb * 8},
                {(void**)&c->order_vals, mb * 4},
                {(void**)&c->ctl_i, 4 * sizeof(int32_t)},
                {(void**)&c->ctl_d, 4 * sizeof(double)}};
    for (auto& r : reqs) {
        if (cudaMalloc(r.ptr, r.bytes) != cudaSuccess) {
            cudaGetLastError();
            free_all(c);
            delete c;
            return DENSER_ERR_CUDA;
        }
    }
    if (cudaMallocHost((void**)&c->h_counters, kNumCounters * 4) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_energy, 2 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_ctl_i, 4 * sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_ctl_d, 4 * sizeof(double)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->dstage_copied[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->dstage_copied[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->dstage_free[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->dstage_free[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return DENSER_ERR_CUDA;
    }
    // after the energy partials: 1/(2 lambda w) for the counts w = 1 .. kInvWeights, each an
    // IEEE float64 division, so that the dual energy multiplies where it would divide
    std::vector<double> inv2lw(kInvWeights);
    for (int i = 0; i < kInvWeights; ++i) inv2lw[i] = 1.0 / (2.0 * c->prm.lambda * (double)(i + 1));
    if (cudaMemcpy(c->d.partials + 2 * kEnergyGrid + 2, inv2lw.data(), kInvWeights * sizeof(double),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        configure_kernels(c) != DENSER_OK || denser_reset(c, nullptr) != DENSER_OK ||
        cudaDeviceSynchronize() != cudaSuccess) {
        free_all(c);
        delete c;
        return DENSER_ERR_CUDA;
    }
    *out = c;
    return DENSER_OK;
}

void denser_destroy(denser_ctx* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        cudaDeviceSynchronize();
        free_all(c);
    }
    delete c;
}

int denser_set_fusion_profiling(denser_ctx* c, int32_t enable) {
    return guarded(c, [&]() -> int {
        if (enable && !c->prof_ev[0])
            for (cudaEvent_t& e : c->prof_ev) {
                const int rc = cuda_check(c, cudaEventCreate(&e), "cudaEventCreate(profile)");
                if (rc) return rc;
            }
        c->profile = enable != 0;
        c->prof = denser_fusion_profile{};
        return DENSER_OK;
    });
}

int denser_get_fusion_profile(const denser_ctx* c, denser_fusion_profile* out) {
    if (!c || !out) return DENSER_ERR_INVALID_ARG;
    *out = c->prof;
    return DENSER_OK;
}

int denser_reset(denser_ctx* c, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc;
        if ((rc = cuda_check(c, cudaMemsetAsync(c->d.hash_keys, 0xff, (size_t)c->prm.hash_slots * 8, s), "reset")))
            return rc;
        if ((rc = cuda_check(c, cudaMemsetAsync(c->d.hash_vals, 0xff, (size_t)c->prm.hash_slots * 4, s), "reset")))
            return rc;
        if ((rc = cuda_check(c, cudaMemsetAsync(c->d.hash_birth, 0x7f, (size_t)c->prm.hash_slots * 4, s), "reset")))
            return rc;
        if ((rc = cuda_check(c, cudaMemsetAsync(c->d.counters, 0, kCounterWords * 4, s), "reset"))) return rc;
        c->cur = 0;
        c->nbr_valid_blocks = -1;
        c->order_valid_blocks = -1;
        return DENSER_OK;
    });
}

const char* denser_last_error(const denser_ctx* c) { return c ? c->msg.c_str() : "null context"; }

int denser_sync(denser_ctx* c, void* stream) {
    return guarded(c, [&]() -> int { return read_counters(c, (cudaStream_t)stream); });
}

int denser_alloc_blocks(denser_ctx* c, const float* depth, const denser_intrinsics* K, const double T_gc[16],
                        int32_t segment, void* stream, int32_t* n_new_out) {
    return guarded(c, [&]() -> int {
        if (!depth || !valid_intrinsics(K) || !valid_pose(T_gc) || segment < 0 || segment > kMaxSegment)
            return set_error(c, DENSER_ERR_INVALID_ARG, "alloc_blocks: bad depth, intrinsics, pose or segment");
        cudaStream_t s = (cudaStream_t)stream;
        const float* dd;
        int slot;
        int rc = stage_depth(c, depth, (size_t)K->width * K->height * 4, s, &dd, &slot);
        if (rc) return rc;
        rc = launch_alloc(c, dd, 1, K, T_gc, segment, s);
        const int rr = release_depth(c, slot, s);
        if (rc || (rc = rr)) return rc;
        if (n_new_out) {
            rc = read_counters(c, s);
            *n_new_out = c->h_counters[kLastNew];
            return rc;
        }
        return DENSER_OK;
    });
}

int denser_fuse_depth(denser_ctx* c, const float* depth, const denser_intrinsics* K, const double T_gc[16],
                      int32_t segment, void* stream) {
    return guarded(c, [&]() -> int {
        if (!depth || !valid_intrinsics(K) || !valid_pose(T_gc) || segment < 0 || segment > kMaxSegment)
            return set_error(c, DENSER_ERR_INVALID_ARG, "fuse_depth: bad depth, intrinsics, pose or segment");
        cudaStream_t s = (cudaStream_t)stream;
        const float* dd;
        int slot;
        int rc = stage_depth(c, depth, (size_t)K->width * K->height * 4, s, &dd, &slot);
        if (rc) return rc;
        rc = launch_fuse(c, dd, 1, K, T_gc, segment, s);
        const int rr = release_depth(c, slot, s);
        return rc ? rc : rr;
    });
}

int denser_integrate(denser_ctx* c, const float* depth, const denser_intrinsics* K, const double T_gc[16],
                     int32_t segment, void* stream, int32_t* n_new_out) {
    return guarded(c, [&]() -> int {
        if (!depth || !valid_intrinsics(K) || !valid_pose(T_gc) || segment < 0 || segment > kMaxSegment)
            return set_error(c, DENSER_ERR_INVALID_ARG, "integrate: bad depth, intrinsics, pose or segment");
        cudaStream_t s = (cudaStream_t)stream;
        const float* dd;
        int slot;
        int rc = stage_depth(c, depth, (size_t)K->width * K->height * 4, s, &dd, &slot);
        if (rc) return rc;
        rc = launch_alloc(c, dd, 1, K, T_gc, segment, s);
        if (!rc) rc = launch_fuse(c, dd, 1, K, T_gc, segment, s, true);
        const int rr = release_depth(c, slot, s);
        if (rc || (rc = rr)) return rc;
        if (n_new_out) {
            rc = read_counters(c, s);
            *n_new_out = c->h_counters[kLastNew];
            return rc;
        }
        return DENSER_OK;
    });
}

int denser_integrate_batch(denser_ctx* c, const float* depths, int32_t n_frames, const denser_intrinsics* K,
                           const double* T_gc, int32_t segment, void* stream, int32_t* n_new_out) {
    return guarded(c, [&]() -> int {
        if (!depths || n_frames < 1 || !T_gc || !valid_intrinsics(K) || segment < 0 || segment > kMaxSegment)
            return set_error(c, DENSER_ERR_INVALID_ARG,
                             "integrate_batch: bad depth maps, frame count, intrinsics, poses or segment");
        for (int i = 0; i < n_frames; ++i)
            if (!valid_pose(T_gc + 16 * (size_t)i))
                return set_error(c, DENSER_ERR_INVALID_ARG, "integrate_batch: pose " + std::to_string(i) + " is not finite");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t map_floats = (size_t)K->width * K->height;
        int64_t added = 0;
        for (int first = 0; first < n_frames; first += kMaxBatch) {
            const int n = std::min(kMaxBatch, n_frames - first);
            const float* dd;
            int slot;
            int rc = stage_depth(c, depths + (size_t)first * map_floats, (size_t)n * map_floats * 4, s, &dd, &slot);
            if (rc) return rc;
            rc = launch_alloc(c, dd, n, K, T_gc + 16 * (size_t)first, segment, s);
            if (!rc) rc = launch_fuse(c, dd, n, K, T_gc + 16 * (size_t)first, segment, s, true);
            const int rr = release_depth(c, slot, s);
            if (rc || (rc = rr)) return rc;
            if (c->profile) {
                if ((rc = read_counters(c, s))) return rc;
                float ms[4];
                for (int e = 0; e < 4; ++e)
                    if ((rc = cuda_check(c, cudaEventElapsedTime(&ms[e], c->prof_ev[e], c->prof_ev[e + 1]),
                                         "profile events")))
                        return rc;
                c->prof.groups += 1;
                c->prof.maps += n;
                c->prof.listed_blocks += c->h_counters[kNumVisible];
                c->prof.new_blocks += c->h_counters[kLastNew];
                c->prof.key_pass_ms += ms[0], c->prof.alloc_rest_ms += ms[1];
                c->prof.cull_ms += ms[2], c->prof.fuse_ms += ms[3];
            }
            if (n_new_out) {
                if ((rc = read_counters(c, s))) return rc;
                added += c->h_counters[kLastNew];
            }
        }
        if (n_new_out) *n_new_out = (int32_t)added;
        return DENSER_OK;
    });
}

// Laser scans: points float32 [n][3] in the sensor frame, host or device memory.
static int points_call(denser_ctx* c, const float* points, int64_t n_points, const double T_gs[16], int32_t segment,
                void* stream, int32_t* n_new_out, bool alloc, bool fuse, const char* what) {
    return guarded(c, [&]() -> int {
        if (n_points < 0 || n_points > (1ll << 28) || (n_points > 0 && !points) || !valid_pose(T_gs) || segment < 0 ||
            segment > kMaxSegment)
            return set_error(c, DENSER_ERR_INVALID_ARG, std::string(what) + ": bad points, count, pose or segment");
        cudaStream_t s = (cudaStream_t)stream;
        const float* dp = nullptr;
        int slot = -1, rc;
        if (n_points > 0 && (rc = stage_depth(c, points, (size_t)n_points * 12, s, &dp, &slot))) return rc;
        rc = DENSER_OK;
        if (alloc) rc = launch_alloc_points(c, dp, n_points, T_gs, segment, s);
        if (!rc && fuse) rc = launch_fuse_points(c, dp, n_points, T_gs, segment, s);
        const int rr = release_depth(c, slot, s);
        if (rc || (rc = rr)) return rc;
        if (n_new_out) {
            rc = read_counters(c, s);
            *n_new_out = c->h_counters[kLastNew];
            return rc;
        }
        return DENSER_OK;
    });
}

int denser_alloc_points(denser_ctx* c, const float* points, int64_t n_points, const double T_gs[16], int32_t segment,
                        void* stream, int32_t* n_new_out) {
    return points_call(c, points, n_points, T_gs, segment, stream, n_new_out, true, false, "alloc_points");
}

int denser_fuse_points(denser_ctx* c, const float* points, int64_t n_points, const double T_gs[16], int32_t segment,
                       void* stream) {
    return points_call(c, points, n_points, T_gs, segment, stream, nullptr, false, true, "fuse_points");
}

int denser_integrate_points(denser_ctx* c, const float* points, int64_t n_points, const double T_gs[16],
                            int32_t segment, void* stream, int32_t* n_new_out) {
    return points_call(c, points, n_points, T_gs, segment, stream, n_new_out, true, true, "integrate_points");
}

// ------------------------------------------------------------------ stereo
static bool dev_all(std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (!p || !is_device_ptr(p)) return false;
    return true;
}

static bool stereo_size_ok(int32_t W, int32_t H) {
    return W >= 2 && H >= 2 && (int64_t)W * H < (1ll << 30);
}

void denser_stereo_default_params(denser_stereo_params* p) {
    if (!p) return;
    p->max_disp = 128;
    p->lambda = 0.5f, p->alpha1 = 1.0f, p->alpha2 = 5.0f;
    p->beta = 1.0f, p->gamma = 4.0f;
    p->theta0 = 2.0f, p->theta_decay = 0.5f;
    p->outer = 8, p->inner = 80;
}

int denser_census(const float* img, int32_t W, int32_t H, uint64_t* sig, void* stream) {
    if (!stereo_size_ok(W, H) || !dev_all({img, sig})) return DENSER_ERR_INVALID_ARG;
    return stereo_census(img, W, H, (unsigned long long*)sig, (cudaStream_t)stream);
}

int denser_diffusion_tensor(const float* img, int32_t W, int32_t H, float gamma, float beta, float* T, void* stream) {
    if (!stereo_size_ok(W, H) || !dev_all({img, T}) || !(gamma >= 0) || !(beta > 0)) return DENSER_ERR_INVALID_ARG;
    return stereo_tensor(img, W, H, gamma, beta, T, (cudaStream_t)stream);
}

int denser_disparity_assign(const uint64_t* sigL, const uint64_t* sigR, int32_t W, int32_t H, int32_t D, float lambda,
                            double theta, const float* d, float* a, void* stream) {
    if (!stereo_size_ok(W, H) || D < 1 || D > 4096 || !dev_all({sigL, sigR, d, a}) || !(lambda >= 0))
        return DENSER_ERR_INVALID_ARG;
    return stereo_assign((const unsigned long long*)sigL, (const unsigned long long*)sigR, W, H, D, lambda, theta, d,
                         a, (cudaStream_t)stream);
}

int denser_tgv_iterate(const float* a, const float* T, int32_t W, int32_t H, float alpha1, float alpha2, double theta,
                       int32_t iters, float* state, void* stream) {
    if (!stereo_size_ok(W, H) || iters < 0 || !(alpha1 > 0) || !(alpha2 > 0) || !(theta > 0) ||
        !dev_all({a, T, state}))
        return DENSER_ERR_INVALID_ARG;
    return stereo_tgv(a, T, W, H, alpha1, alpha2, theta, iters, state, (cudaStream_t)stream);
}

size_t denser_stereo_workspace_size(int32_t W, int32_t H) {
    if (!stereo_size_ok(W, H)) return 0;
    // sig_L, sig_R (8 bytes a pixel), tensor (3), a, state (2 x 12) float planes
    return (size_t)W * H * (16 + 4 * 28);
}

int denser_stereo_estimate(const float* IL, const float* IR, int32_t W, int32_t H, const denser_stereo_params* p,
                           void* ws, size_t ws_bytes, float* disparity, void* stream) {
    if (!stereo_size_ok(W, H) || !p || p->max_disp < 1 || p->max_disp > 4096 || p->outer < 0 || p->inner < 0 ||
        !(p->theta0 > 0) || !(p->theta_decay > 0) || !(p->alpha1 > 0) || !(p->alpha2 > 0) || !(p->lambda >= 0) ||
        !(p->gamma >= 0) || !(p->beta > 0) || ws_bytes < denser_stereo_workspace_size(W, H) ||
        !dev_all({IL, IR, ws, disparity}))
        return DENSER_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)W * H;
    unsigned long long* sigL = (unsigned long long*)ws;
    unsigned long long* sigR = sigL + n;
    float* T = (float*)(sigR + n);
    float* a = T + 3 * n;
    float* state = a + n;
    int rc;
    if ((rc = stereo_census(IL, W, H, sigL, s)) || (rc = stereo_census(IR, W, H, sigR, s)) ||
        (rc = stereo_tensor(IR, W, H, p->gamma, p->beta, T, s)))
        return rc;
    if (cudaMemsetAsync(a, 0, n * 4, s) != cudaSuccess) return DENSER_ERR_CUDA;
    // start: winner takes all (no coupling), w = p = q = 0
    if ((rc = stereo_assign(sigL, sigR, W, H, p->max_disp, p->lambda, 0.0, a, a, s)) ||
        (rc = stereo_init_state(state, a, W, H, s)))
        return rc;
    double theta = p->theta0;
    for (int k = 0; k < p->outer; ++k) {
        if ((rc = stereo_assign(sigL, sigR, W, H, p->max_disp, p->lambda, theta, state, a, s)) ||
            (rc = stereo_tgv(a, T, W, H, p->alpha1, p->alpha2, theta, p->inner, state, s)))
            return rc;
        theta *= p->theta_decay;
    }
    return cudaMemcpyAsync(disparity, state, n * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? DENSER_OK
                                                                                               : DENSER_ERR_CUDA;
}

int denser_disparity_to_depth(const float* disp, int32_t W, int32_t H, float fx, float baseline, float min_disp,
                              float* depth, void* stream) {
    if (!stereo_size_ok(W, H) || !(fx > 0) || !(baseline > 0) || !(min_disp >= 0) || !dev_all({disp, depth}))
        return DENSER_ERR_INVALID_ARG;
    return stereo_depth(disp, W, H, fx * baseline, min_disp, depth, (cudaStream_t)stream);
}

int denser_regularize(denser_ctx* c, int32_t max_iters, double gap_tol, int32_t start, void* stream,
                      denser_reg_stats* out) {
    return guarded(c, [&]() -> int {
        if (max_iters < 0 || !(gap_tol >= 0) || (start != 0 && start != 1))
            return set_error(c, DENSER_ERR_INVALID_ARG, "regularize: bad max_iters, gap_tol or start");
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        const size_t nv = (size_t)nb * kBlockVoxels;
        const size_t pstride_bytes = (size_t)c->d.max_blocks * kBlockVoxels * c->elem_size;
        cudaEvent_t e0, e1, a0, a1;
        cudaEventCreate(&e0), cudaEventCreate(&e1), cudaEventCreate(&a0), cudaEventCreate(&a1);
        struct EvFree {
            cudaEvent_t* e;
            ~EvFree() {
                for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
            }
        };
        cudaEvent_t evs[4] = {e0, e1, a0, a1};
        EvFree ef{evs};
        cudaEventRecord(e0, s);
        rc = launch_prepare_regularize(c, nb, c->nbr_valid_blocks != nb, s);
        if (rc) return rc;
        if (start == 0 && nb > 0) {
            rc = cuda_check(c, cudaMemsetAsync(c->d.u, 0, nv * c->elem_size, s), "zero u");
            if (!rc) rc = cuda_check(c, cudaMemsetAsync(c->d.ub[c->cur], 0, nv * c->elem_size, s), "zero u_bar");
            for (int a = 0; a < 3 && !rc; ++a)
                rc = cuda_check(c, cudaMemsetAsync((char*)c->d.p[c->cur] + a * pstride_bytes, 0, nv * c->elem_size, s),
                                "zero p");
            if (rc) return rc;
        }
        const bool check_gap = gap_tol > 0 && c->prm.gap_every > 0;
        double sweep_ms = 0.0;
        int launches = 0, gap_evals = 0, converged = 0, it = 0;
        double P = NAN, D = NAN;
        bool have_energy = false;
        // graph-captured body passes of k iterations (k even keeps the ping-pong parity)
        const int k = check_gap ? c->prm.gap_every : 10;
        if (c->sched.use_graph && nb > 0 && k % 2 == 0 && max_iters >= k) {
            c->h_ctl_i[0] = 0, c->h_ctl_i[1] = max_iters, c->h_ctl_i[2] = 0, c->h_ctl_i[3] = 0;
            c->h_ctl_d[0] = gap_tol, c->h_ctl_d[1] = c->h_ctl_d[2] = c->h_ctl_d[3] = 0.0;
            rc = cuda_check(c, cudaMemcpyAsync(c->ctl_i, c->h_ctl_i, 4 * sizeof(int32_t), cudaMemcpyHostToDevice, s),
                            "loop control");
            if (!rc)
                rc = cuda_check(c, cudaMemcpyAsync(c->ctl_d, c->h_ctl_d, 4 * sizeof(double), cudaMemcpyHostToDevice, s),
                                "loop control");
            if (!rc) rc = cuda_check(c, cudaEventRecord(a0, s), "event");
            if (!rc) rc = launch_graph_loop(c, nb, k, check_gap, s);
            if (!rc) rc = cuda_check(c, cudaEventRecord(a1, s), "event");
            if (rc) return rc;
            if (check_gap || out) {
                rc = cuda_check(c, cudaMemcpyAsync(c->h_ctl_i, c->ctl_i, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                                "loop control");
                if (!rc)
                    rc = cuda_check(c, cudaMemcpyAsync(c->h_ctl_d, c->ctl_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, s),
                                    "loop control");
                if (!rc) rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
                if (rc) return rc;
                it = c->h_ctl_i[0];
                converged = c->h_ctl_i[2];
                gap_evals = c->h_ctl_i[3];
                if (gap_evals > 0) P = c->h_ctl_d[1], D = c->h_ctl_d[2], have_energy = true;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a0, a1);
                sweep_ms += ms;
            } else {
                it = (max_iters / k) * k;  // without gap checks the pass count is fixed
            }
            launches += it;
            c->launches += (unsigned long long)(it / k) * (k + (check_gap ? 2 : 0) + 1);
        }
        while (it < max_iters && !converged) {
            int batch = max_iters - it;
            if (check_gap) batch = std::min(batch, c->prm.gap_every - (it % c->prm.gap_every));
            cudaEventRecord(a0, s);
            for (int k = 0; k < batch; ++k) {
                rc = launch_sweep(c, nb, s);
                if (rc) return rc;
            }
            cudaEventRecord(a1, s);
            it += batch;
            launches += nb > 0 ? batch : 0;
            const bool gap_due = check_gap && it % c->prm.gap_every == 0;
            if (gap_due || out) {
                // events complete once the stream reaches them
                if ((rc = cuda_check(c, cudaEventSynchronize(a1), "event synchronize"))) return rc;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a0, a1);
                sweep_ms += ms;
            }
            if (gap_due) {
                if ((rc = energy_now(c, nb, s, &P, &D))) return rc;
                have_energy = true;
                ++gap_evals;
                if ((P - D) <= gap_tol * fabs(P)) {
                    converged = 1;
                    break;
                }
            } else {
                have_energy = false;
            }
        }
        if (out) {
            if (!have_energy && (rc = energy_now(c, nb, s, &P, &D))) return rc;
            cudaEventRecord(e1, s);
            if ((rc = read_counters(c, s))) return rc;
            float tot = 0.f;
            cudaEventElapsedTime(&tot, e0, e1);
            memset(out, 0, sizeof(*out));
            out->iters = it;
            out->converged = converged || (gap_tol > 0 && (P - D) <= gap_tol * fabs(P));
            out->primal = P;
            out->dual = D;
            out->gap = P - D;
            out->rel_gap = P != 0 ? (P - D) / fabs(P) : 0.0;
            out->sweep_ms = sweep_ms;
            out->total_ms = tot;
            out->sweep_launches = launches;
            out->gap_evals = gap_evals;
            out->n_blocks = nb;
            out->n_omega = -1;
        }
        return DENSER_OK;
    });
}

int denser_energy(denser_ctx* c, double* primal, double* dual, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if ((rc = launch_prepare_regularize(c, nb, c->nbr_valid_blocks != nb, s))) return rc;
        double P, D;
        if ((rc = energy_now(c, nb, s, &P, &D))) return rc;
        if (primal) *primal = P;
        if (dual) *dual = D;
        return DENSER_OK;
    });
}

int denser_extract(denser_ctx* c, int32_t* coords, float* f, float* w, uint8_t* omega, float* u,
                   int64_t capacity_blocks, int64_t* n_blocks_out, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if (n_blocks_out) *n_blocks_out = nb;
        if ((coords || f || w || omega || u) && capacity_blocks < nb)
            return set_error(c, DENSER_ERR_INVALID_ARG, "extract: capacity_blocks < number of blocks");
        const size_t nv = (size_t)nb * kBlockVoxels;
        if (nb == 0) return DENSER_OK;
        if (coords && (rc = copy_out(c, coords, c->d.coords, (size_t)nb * 16, s, "copy coords"))) return rc;
        if (f && (rc = copy_out(c, f, c->d.f, nv * 4, s, "copy f"))) return rc;
        if (w && (rc = copy_out(c, w, c->d.w, nv * 4, s, "copy w"))) return rc;
        if (u && (rc = copy_state_out(c, u, c->d.u, (int64_t)nv, s))) return rc;
        if (omega) {
            uint8_t* dst = omega;
            if (!is_device_ptr(omega)) {
                if ((rc = ensure_conv(c, nv))) return rc;
                dst = (uint8_t*)c->conv_scratch;
            }
            if ((rc = launch_omega_bytes(c, nb, dst, s))) return rc;
            if (dst != omega && (rc = copy_out(c, omega, dst, nv, s, "copy omega"))) return rc;
        }
        return cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
    });
}

int denser_extract_dual(denser_ctx* c, float* u_bar, float* p, int64_t capacity_blocks, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if ((u_bar || p) && capacity_blocks < nb)
            return set_error(c, DENSER_ERR_INVALID_ARG, "extract_dual: capacity_blocks < number of blocks");
        const int64_t nv = nb * kBlockVoxels;
        if (nb == 0) return DENSER_OK;
        if (u_bar && (rc = copy_state_out(c, u_bar, c->d.ub[c->cur], nv, s))) return rc;
        if (p) {
            const size_t pstride = (size_t)c->d.max_blocks * kBlockVoxels * c->elem_size;
            for (int a = 0; a < 3; ++a)
                if ((rc = copy_state_out(c, p + a * nv, (char*)c->d.p[c->cur] + a * pstride, nv, s))) return rc;
        }
        return cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
    });
}

int denser_extract_surface(denser_ctx* c, float* tri_pos, int64_t* tri_ids, int64_t capacity, int64_t* n_tri_out,
                           int64_t* block_first, void* stream) {
    return guarded(c, [&]() -> int {
        if (!n_tri_out || capacity < 0)
            return set_error(c, DENSER_ERR_INVALID_ARG, "extract_surface: n_tri_out is required and capacity >= 0");
        *n_tri_out = 0;
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if (nb == 0) {
            if (block_first) {  // host or device memory: written through a copy
                const long long zero = 0;
                if ((rc = copy_out(c, block_first, &zero, 8, s, "copy block offsets"))) return rc;
                return cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
            }
            return DENSER_OK;
        }
        if (!c->surf_counts) {
            if ((rc = cuda_check(c, cudaMalloc(&c->surf_counts, (size_t)c->d.max_blocks * 4), "cudaMalloc(surface counts)")))
                return rc;
            if ((rc = cuda_check(c, cudaMalloc(&c->surf_offsets, ((size_t)c->d.max_blocks + 1) * 8),
                                 "cudaMalloc(surface offsets)")))
                return rc;
            if ((rc = cuda_check(c, cudaMalloc(&c->surf_up, (size_t)c->d.max_blocks * 32), "cudaMalloc(surface neighbours)")))
                return rc;
            if ((rc = cuda_check(c, cudaMalloc(&c->surf_cursor, 8), "cudaMalloc(surface cursor)"))) return rc;
        }
        long long total = 0;
        unsigned long long items = 0;
        const bool device_out = (!tri_pos || is_device_ptr(tri_pos)) && (!tri_ids || is_device_ptr(tri_ids));
        if ((tri_pos || tri_ids) && device_out && capacity > 0) {
            // device outputs: count, scan and emit queued back to back, one wait at the end;
            // a list that overflowed (the emit then wrote nothing) is grown and both redone
            for (int attempt = 0; attempt < 2; ++attempt) {
                const long long need = attempt == 0 ? std::max<long long>((long long)nb * 32, c->surf_list_cap)
                                                    : (long long)items;
                if (c->surf_list_cap < need) {
                    if (c->surf_list) cudaFree(c->surf_list);
                    c->surf_list = nullptr;
                    c->surf_list_cap = 0;
                    if ((rc = cuda_check(c, cudaMalloc(&c->surf_list, (size_t)need * 8), "cudaMalloc(surface list)")))
                        return rc;
                    c->surf_list_cap = need;
                }
                if ((rc = launch_surface(c, nb, 0, nullptr, nullptr, 0, s))) return rc;
                if ((rc = launch_surface(c, nb, 2, tri_pos, (long long*)tri_ids, capacity, s))) return rc;
                if ((rc = copy_out(c, &total, c->surf_offsets + nb, 8, s, "read triangle count"))) return rc;
                if ((rc = copy_out(c, &items, c->surf_cursor, 8, s, "read cube count"))) return rc;
                if ((rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize"))) return rc;
                if ((long long)items <= c->surf_list_cap) break;
            }
            c->surf_items = (long long)items;
            *n_tri_out = total;
            if (block_first) {
                if ((rc = copy_out(c, block_first, c->surf_offsets, ((size_t)nb + 1) * 8, s, "copy block offsets")))
                    return rc;
                if ((rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize"))) return rc;
            }
            if (total > capacity)
                return set_error(c, DENSER_ERR_TOO_LARGE,
                                 "extract_surface: more triangles than capacity (*n_tri_out holds the total)");
            return DENSER_OK;
        }
        for (int attempt = 0; attempt < 2; ++attempt) {
            // first a guess of 32 listed cubes per block, then exactly what the count found
            const long long need = attempt == 0 ? (long long)nb * 32 : (long long)items;
            if (c->surf_list_cap < need) {
                if (c->surf_list) cudaFree(c->surf_list);
                c->surf_list = nullptr;
                c->surf_list_cap = 0;
                if ((rc = cuda_check(c, cudaMalloc(&c->surf_list, (size_t)need * 8), "cudaMalloc(surface list)")))
                    return rc;
                c->surf_list_cap = need;
            }
            if ((rc = launch_surface(c, nb, 0, nullptr, nullptr, 0, s))) return rc;
            if ((rc = copy_out(c, &total, c->surf_offsets + nb, 8, s, "read triangle count"))) return rc;
            if ((rc = copy_out(c, &items, c->surf_cursor, 8, s, "read cube count"))) return rc;
            if ((rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize"))) return rc;
            if ((long long)items <= c->surf_list_cap) break;  // else grow to the exact need and count again
        }
        c->surf_items = (long long)items;
        *n_tri_out = total;
        if (block_first && (rc = copy_out(c, block_first, c->surf_offsets, ((size_t)nb + 1) * 8, s, "copy block offsets")))
            return rc;
        if (!tri_pos && !tri_ids) return cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
        const int64_t n_out = std::min<int64_t>(total, capacity);
        if (n_out > 0) {
            // host outputs go through device scratch: ids first (8-byte aligned), then positions
            const bool host_ids = tri_ids && !is_device_ptr(tri_ids), host_pos = tri_pos && !is_device_ptr(tri_pos);
            const size_t ids_bytes = (size_t)n_out * 24, pos_bytes = (size_t)n_out * 36;
            const size_t need = (host_ids ? ids_bytes : 0) + (host_pos ? pos_bytes : 0);
            if (need > c->surf_bytes) {
                if (c->surf_scratch) cudaFree(c->surf_scratch);
                c->surf_scratch = nullptr;
                c->surf_bytes = 0;
                if ((rc = cuda_check(c, cudaMalloc(&c->surf_scratch, need), "cudaMalloc(surface scratch)"))) return rc;
                c->surf_bytes = need;
            }
            long long* dids = host_ids ? (long long*)c->surf_scratch : (long long*)tri_ids;
            float* dpos = host_pos ? (float*)((char*)c->surf_scratch + (host_ids ? ids_bytes : 0)) : tri_pos;
            if ((rc = launch_surface(c, nb, 1, dpos, dids, n_out, s))) return rc;
            if (host_ids && (rc = copy_out(c, tri_ids, dids, ids_bytes, s, "copy triangle ids"))) return rc;
            if (host_pos && (rc = copy_out(c, tri_pos, dpos, pos_bytes, s, "copy triangles"))) return rc;
        }
        if ((rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize"))) return rc;
        if (total > capacity)
            return set_error(c, DENSER_ERR_TOO_LARGE,
                             "extract_surface: more triangles than capacity (*n_tri_out holds the total)");
        return DENSER_OK;
    });
}

int denser_load_blocks(denser_ctx* c, const int32_t* coords, const float* f, const float* w, int64_t n,
                       void* stream) {
    return guarded(c, [&]() -> int {
        if (n < 0 || (n > 0 && !coords)) return set_error(c, DENSER_ERR_INVALID_ARG, "load_blocks: bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t base = c->h_counters[kNumBlocks];
        if (base + n > (int64_t)c->d.max_blocks)
            return set_error(c, DENSER_ERR_POOL_FULL, "load_blocks: more blocks than max_blocks");
        if (n == 0) return DENSER_OK;
        const void* cd;
        if ((rc = device_input(c, coords, (size_t)n * 16, s, &cd))) return rc;
        if ((rc = launch_load_blocks(c, (const int32_t*)cd, n, base, s))) return rc;
        const size_t nv = (size_t)n * kBlockVoxels;
        if (f && (rc = copy_out(c, c->d.f + (size_t)base * kBlockVoxels, f, nv * 4, s, "copy f in"))) return rc;
        if (w && (rc = copy_out(c, c->d.w + (size_t)base * kBlockVoxels, w, nv * 4, s, "copy w in"))) return rc;
        return read_counters(c, s);
    });
}

int denser_load_state(denser_ctx* c, const float* u, const float* u_bar, const float* p, int64_t n, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if (n != nb) return set_error(c, DENSER_ERR_INVALID_ARG, "load_state: n must equal the number of blocks");
        if (nb == 0) return DENSER_OK;
        const int64_t nv = nb * kBlockVoxels;
        if ((rc = copy_state_in(c, c->d.u, u, nv, s))) return rc;
        if ((rc = copy_state_in(c, c->d.ub[c->cur], u_bar, nv, s))) return rc;
        const size_t pstride = (size_t)c->d.max_blocks * kBlockVoxels * c->elem_size;
        for (int a = 0; a < 3; ++a)
            if ((rc = copy_state_in(c, (char*)c->d.p[c->cur] + a * pstride, p ? p + a * nv : nullptr, nv, s)))
                return rc;
        return read_counters(c, s);
    });
}

// ------------------------------------------------------------- warm start
namespace {
int net_blocks_check(denser_ctx* c, const int32_t* blocks, int64_t n, int64_t nb) {
    if (n < 0 || n > nb || (n > 0 && blocks && !is_device_ptr(blocks)))
        return set_error(c, DENSER_ERR_INVALID_ARG, "net: n out of range or block list not in device memory");
    return DENSER_OK;
}
}  // namespace

int denser_net_gather(denser_ctx* c, const int32_t* blocks, int64_t n, void* x, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        if ((rc = net_blocks_check(c, blocks, n, c->h_counters[kNumBlocks]))) return rc;
        if (n == 0) return DENSER_OK;
        if (!x || !is_device_ptr(x)) return set_error(c, DENSER_ERR_INVALID_ARG, "net_gather: x must be device memory");
        return launch_net_gather(c, blocks, (int)n, x, s);
    });
}

int denser_net_targets_div(denser_ctx* c, const int32_t* blocks, int64_t n, float* target, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if ((rc = net_blocks_check(c, blocks, n, nb))) return rc;
        if (n == 0) return DENSER_OK;
        if (!target || !is_device_ptr(target))
            return set_error(c, DENSER_ERR_INVALID_ARG, "net_targets_div: target must be device memory");
        if ((rc = launch_prepare_regularize(c, nb, c->nbr_valid_blocks != nb, s))) return rc;
        return launch_net_targets_div(c, blocks, (int)n, target, s);
    });
}

int denser_net_targets(denser_ctx* c, const int32_t* blocks, int64_t n, float* target, float* mask, float u_weight,
                       float p_weight, void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if ((rc = net_blocks_check(c, blocks, n, nb))) return rc;
        if (n == 0) return DENSER_OK;
        if (!target || !mask || !is_device_ptr(target) || !is_device_ptr(mask) || !(u_weight >= 0) || !(p_weight >= 0))
            return set_error(c, DENSER_ERR_INVALID_ARG, "net_targets: outputs must be device memory, weights >= 0");
        if ((rc = launch_prepare_regularize(c, nb, c->nbr_valid_blocks != nb, s))) return rc;
        return launch_net_targets(c, blocks, (int)n, target, mask, sqrtf(u_weight), sqrtf(p_weight), s);
    });
}

int denser_net_apply(denser_ctx* c, const int32_t* blocks, int64_t n, const float* out, int32_t with_dual,
                     void* stream) {
    return guarded(c, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = read_counters(c, s);
        if (rc) return rc;
        const int64_t nb = c->h_counters[kNumBlocks];
        if ((rc = net_blocks_check(c, blocks, n, nb))) return rc;
        if (n == 0) return DENSER_OK;
        if (!out || !is_device_ptr(out)) return set_error(c, DENSER_ERR_INVALID_ARG, "net_apply: out must be device memory");
        if (with_dual < 0 || with_dual > 2) return set_error(c, DENSER_ERR_INVALID_ARG, "net_apply: with_dual must be 0, 1 or 2");
        if ((rc = launch_prepare_regularize(c, nb, c->nbr_valid_blocks != nb, s))) return rc;
        return launch_net_apply(c, blocks, (int)n, out, with_dual, s);
    });
}

int denser_set_schedule(denser_ctx* c, const denser_schedule* sch) {
    if (!c || !sch) return DENSER_ERR_INVALID_ARG;
    if (sch->sweep_kernel < 0 || sch->sweep_kernel > 9 || sch->order < 0 || sch->order > 1 || sch->ctas_per_sm < 0 ||
        sch->ctas_per_sm > 8 || sch->use_graph < 0 || sch->use_graph > 1)
        return set_error(c, DENSER_ERR_INVALID_ARG, "set_schedule: field out of range");
    c->sched = *sch;
    c->order_valid_blocks = -1;
    return DENSER_OK;
}

int denser_get_schedule(const denser_ctx* c, denser_schedule* sch) {
    if (!c || !sch) return DENSER_ERR_INVALID_ARG;
    *sch = c->sched;
    return DENSER_OK;
}

int64_t denser_num_blocks(denser_ctx* c, void* stream) {
    if (!c) return DENSER_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    int rc = read_counters(c, (cudaStream_t)stream);
    if (rc) return rc;
    return c->h_counters[kNumBlocks];
}

uint64_t denser_launch_count(const denser_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
