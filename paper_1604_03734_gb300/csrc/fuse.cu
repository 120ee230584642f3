// Projective TSDF fusion, Eq. 1 (Section III-A, steps 1-4).
//
// One fusion call takes n_frames depth maps of one camera (1..kMaxBatch) in order:
//   depth_max   largest valid depth of each map, unless the allocation of the same maps
//               recorded it (it bounds the blocks that can change);
//   cull        one thread per allocated block tests it against every map: bounding
//               sphere of the voxel centres against the camera's near plane, the viewing
//               frustum's four side planes and the far limit d_max + mu.  Blocks that
//               pass for at least one map go to a work list with the mask of those maps.
//               A culled (block, map) provably has no voxel that Eq. 1 would update.
//               After a batched allocation a block that the batch added takes only the
//               maps from the first one that allocated it on, as one call per map would;
//   origin      the float64 camera-frame origin of each listed (block, map) pair, as a
//               float32 hi/lo pair with its bound, and one bound on the projection error
//               that every voxel of the pair can use (none for blocks that reach too
//               close to the camera plane);
//   fuse        one CTA per listed block, 128 threads x 4 consecutive voxels; f and w
//               stay in registers while the block takes its maps in order, so they move
//               once per call as float4.  Each integer decision (the pixel a voxel
//               projects to, z_c > 0, u_SDF >= -mu) is first taken in float32 together
//               with a forward error bound (the pair's shared projection bound, else the
//               voxel's own); when the bound cannot certify it, the voxel is
//               recomputed in float64 in the oracle's exact operation order.  So the set
//               of updated voxels (and w) is bit-exact while float64, which runs at a
//               small fraction of the float32 rate on this GPU, is used for well under
//               1% of voxels.  f is accumulated in float32, each voxel's maps in order,
//               with the same operations as one call per map.
#include <math.h>

#include "common.cuh"

namespace denser {

namespace {

// The pose of one depth map of the call.
struct FuseFrame {
    double Ri[9];          // R^T
    double ti[3];          // -R^T t
    float M[9];            // s R^T: camera-frame step per local voxel index (float32)
    float Rif[9], tif[3];  // R^T and -R^T t as float32 (the culling test)
    float tabs;            // |t|_1 of -R^T t
};

struct FuseArgs {
    double fx, fy, cx, cy, s, mu;
    double radius;  // bounding-sphere radius of a block's voxel centres, padded
    float fxf, fyf, cxf, cyf, muf, sf, Wf, Hf;
    float imuf;                // 1 / mu as float32
    float planef[4][3];        // unit normals of the four side planes (camera frame), float32
    int W, H, seg, n_frames;
    int gate;                  // blocks the batch added take maps from their birth on
    FuseFrame fr[kMaxBatch];
};

// A listed block and the maps it takes.
struct VisEntry {
    int b;
    uint32_t mask;
};

// The camera-frame centre of a block's voxel (0,0,0) for one map, split into float32
// high and low parts (hi + lo = the float64 value to ~2^-48).
struct VisOrigin {
    float hi[3];
    float lo[3];
    float delta;   // bound on |c0 - (hi + lo)| for the block
    float ex, ey;  // bounds on every voxel's projection error (pixels); ex < 0: none
    float pad[3];
};
static_assert(sizeof(VisOrigin) == 4 * kVisOriginFloats, "fusion origin entry size");

__global__ void __launch_bounds__(256) depth_max_kernel(const float* __restrict__ depth, int n, int32_t* out) {
    __shared__ float red[8];
    float mx = 0.0f;
    const int n4 = ((reinterpret_cast<uintptr_t>(depth) & 15) == 0) ? n / 4 : 0;
    const float4* d4 = reinterpret_cast<const float4*>(depth);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
        const float4 v = __ldg(d4 + i);
        if (isfinite(v.x)) mx = fmaxf(mx, v.x);
        if (isfinite(v.y)) mx = fmaxf(mx, v.y);
        if (isfinite(v.z)) mx = fmaxf(mx, v.z);
        if (isfinite(v.w)) mx = fmaxf(mx, v.w);
    }
    for (int i = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float d = __ldg(depth + i);
        if (isfinite(d)) mx = fmaxf(mx, d);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmaxf(mx, red[i]);
        if (mx > 0.0f) atomicMax(out, __float_as_int(mx));
    }
}

__device__ inline void to_camera(const FuseFrame& fr, double gx, double gy, double gz, double* c) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        c[r] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(fr.Ri[3 * r], gx), __dmul_rn(fr.Ri[3 * r + 1], gy)),
                                   __dmul_rn(fr.Ri[3 * r + 2], gz)),
                         fr.ti[r]);
}

// Bounds on the projection error (pixels, per image axis) shared by the 512 voxels of a
// (block, map) pair, in float32 with every operation rounded explicitly, or -1 when the
// block reaches too close to the camera plane to share them.  It dominates the bound the
// fusion kernel's per-voxel path computes, so the decisions it certifies are the
// float64 ones by the same argument; a larger bound only sends more voxels to float64.
// Per axis r, the float32 coordinate of voxel l is (hi_r + (M_r . l)) + lo_r with
// 0 <= l <= 7, so its magnitude is at most X_r = (|hi_r| + |lo_r| + 7 sum_j |M_rj|)
// (1 + 2^-20) (the factor covers the roundings of both sides), which bounds the
// per-voxel coordinate bound 2^-22 (|x| + 25 s) + delta.  Every voxel's z is at least
// zlo = (hi_z + lo_z) + 7 sum_j min(M_zj, 0) - 2^-21 X_z; when zlo exceeds the z bound,
// every voxel is certainly in front of the camera, its 1/(z - dz) is below
// 1/(zlo - dz) and its |x / z| below X_x / zlo, and the bound follows from the
// per-voxel formulas with those maxima (the final factor covers a different
// contraction of their products into fused multiply-adds).
__device__ inline void shared_projection_bound(const FuseArgs& a, const FuseFrame& fr, const float* hi,
                                               const float* lo, float delta, float* bx, float* by) {
    const float eps22 = 2.38418579e-7f, up = 1.00000095f;  // 2^-22; 1 + 2^-20 rounded up
    const float s25 = __fmul_rn(25.0f, a.sf);
    float X[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float ext = __fmul_rn(7.0f, __fadd_rn(__fadd_rn(fabsf(fr.M[3 * r]), fabsf(fr.M[3 * r + 1])),
                                                  fabsf(fr.M[3 * r + 2])));
        X[r] = __fmul_rn(__fadd_rn(__fadd_rn(fabsf(hi[r]), fabsf(lo[r])), ext), up);
    }
    const float dxb = __fmaf_rn(eps22, __fadd_rn(X[0], s25), delta);
    const float dyb = __fmaf_rn(eps22, __fadd_rn(X[1], s25), delta);
    const float dzb = __fmaf_rn(eps22, __fadd_rn(X[2], s25), delta);
    const float mneg = __fmul_rn(7.0f, __fadd_rn(__fadd_rn(fminf(fr.M[6], 0.0f), fminf(fr.M[7], 0.0f)),
                                               fminf(fr.M[8], 0.0f)));
    const float zlo = __fsub_rn(__fadd_rn(__fadd_rn(hi[2], lo[2]), mneg), __fmul_rn(4.76837158e-7f, X[2]));
    const float gap = __fsub_rn(zlo, dzb);
    *bx = *by = -1.0f;
    if (!(gap > 1.0e-30f)) return;
    const float izb = __fmul_rn(rcp_approx(gap), up);
    const float izl = __fmul_rn(rcp_approx(zlo), up);
    const float rxb = __fmul_rn(__fmul_rn(X[0], izl), up), ryb = __fmul_rn(__fmul_rn(X[1], izl), up);
    const float cx = fabsf(a.cxf), cy = fabsf(a.cyf);
    const float pxb = __fmul_rn(__fmaf_rn(a.fxf, rxb, cx), up), pyb = __fmul_rn(__fmaf_rn(a.fyf, ryb, cy), up);
    const float eps23 = 1.19209290e-7f;  // 2^-23
    const float ex = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(__fmul_rn(a.fxf, __fmaf_rn(rxb, dzb, dxb)), izb), 1.01f),
                                         __fadd_rn(__fmul_rn(eps22, __fmul_rn(a.fxf, rxb)),
                                                   __fmul_rn(eps23, __fadd_rn(pxb, cx)))),
                               1e-6f);
    const float ey = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(__fmul_rn(a.fyf, __fmaf_rn(ryb, dzb, dyb)), izb), 1.01f),
                                         __fadd_rn(__fmul_rn(eps22, __fmul_rn(a.fyf, ryb)),
                                                   __fmul_rn(eps23, __fadd_rn(pyb, cy)))),
                               1e-6f);
    *bx = __fmul_rn(ex, up);
    *by = __fmul_rn(ey, up);
}

// The float64 origin of block key k for map `fr`, as float32 hi + lo with its bound.
__device__ inline VisOrigin block_origin(const FuseArgs& a, const FuseFrame& fr, int4 k) {
    double c0[3];
    to_camera(fr, __dmul_rn(__dadd_rn((double)(8 * k.y), 0.5), a.s), __dmul_rn(__dadd_rn((double)(8 * k.z), 0.5), a.s),
              __dmul_rn(__dadd_rn((double)(8 * k.w), 0.5), a.s), c0);
    VisOrigin o;
    double amax = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        o.hi[e] = (float)c0[e];
        o.lo[e] = (float)(c0[e] - (double)o.hi[e]);
        amax = fmax(amax, fabs(c0[e]));
    }
    // What hi + lo misses of the float64 origin, and the float64 roundings of the
    // oracle's own transform (relative 2^-51 of |R| |g| + |t| per coordinate); the
    // float32 rounding of each voxel's coordinate is bounded per voxel in the fusion.
    const double gmax = (8.0 * (fabs((double)k.y) + fabs((double)k.z) + fabs((double)k.w)) + 24.0) * a.s;
    const double tmax = fabs(fr.ti[0]) + fabs(fr.ti[1]) + fabs(fr.ti[2]);
    o.delta = (float)(ldexp(amax + gmax + tmax + 1.0, -44));
    shared_projection_bound(a, fr, o.hi, o.lo, o.delta, &o.ex, &o.ey);
    o.pad[0] = o.pad[1] = o.pad[2] = 0.0f;
    return o;
}

__global__ void cull_kernel(DeviceMap m, FuseArgs a) {
    const int nb = m.counters[kNumBlocks];
    // blocks [first_new, nb) were added by the batch's allocation
    const int first_new = a.gate ? nb - m.counters[kLastNew] : nb;
    const int lane = threadIdx.x & 31;
    // warp-uniform loop bound: every lane reaches the ballot
    for (int base = blockIdx.x * blockDim.x; base < nb; base += gridDim.x * blockDim.x) {
        const int b = base + (int)threadIdx.x;
        uint32_t mask = 0u;
        if (b < nb) {
            const int4 k = reinterpret_cast<const int4*>(m.coords)[b];
            if (k.x == a.seg) {
                // centre of the block's voxel centres: voxel index 8 b + 3.5 -> (8 b + 4) s.
                // The test only skips blocks that no voxel of can be updated, so float32
                // with a margin is enough: the float32 centre and plane distances are
                // within 2^-21 (|g|_1 + |t|_1 + 1) of the exact ones, the margin is twice that.
                const float gx = (float)(8 * k.y + 4) * a.sf, gy = (float)(8 * k.z + 4) * a.sf,
                            gz = (float)(8 * k.w + 4) * a.sf;
                const float g1 = fabsf(gx) + fabsf(gy) + fabsf(gz) + 1.0f;
                const int from = b >= first_new ? (int)m.block_birth[b] : 0;
                for (int i = from; i < a.n_frames; ++i) {
                    const int dbits = m.counters[kFrameDepthMax + i];
                    if (dbits == 0) continue;  // no valid pixel: nothing can change
                    const float farf = (float)((double)__int_as_float(dbits) + a.mu) * (1.0f + 1.0e-6f) + 1.0e-6f;
                    const FuseFrame& fr = a.fr[i];
                    float c[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        c[r] = fmaf(fr.Rif[3 * r], gx, fmaf(fr.Rif[3 * r + 1], gy, fmaf(fr.Rif[3 * r + 2], gz, fr.tif[r])));
                    const float r = (float)a.radius + 9.53674316e-7f * (g1 + fr.tabs);
                    bool keep = c[2] + r >= 0.0f && c[2] - r <= farf;  // not all behind, not all beyond d + mu
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        keep &= fmaf(a.planef[q][0], c[0], fmaf(a.planef[q][1], c[1], a.planef[q][2] * c[2])) >= -r;
                    if (keep) mask |= 1u << i;
                }
            }
        }
        // one atomic per warp for the work-list slots
        const unsigned ball = __ballot_sync(0xffffffffu, mask != 0u);
        int first = 0;
        if (lane == 0 && ball) first = atomicAdd(m.counters + kNumVisible, __popc(ball));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (mask) {
            VisEntry e;
            e.b = b, e.mask = mask;
            reinterpret_cast<VisEntry*>(m.visible)[first + __popc(ball & ((1u << lane) - 1))] = e;
        }
    }
}

// The float64 origin of every listed (block, map) pair, one thread per pair: the float64
// pipe of this GPU is narrow, so the chains run side by side instead of one map after
// another in the culling thread.
__global__ void __launch_bounds__(256) origin_kernel(DeviceMap m, FuseArgs a) {
    const long long n = (long long)m.counters[kNumVisible] * a.n_frames;
    const VisEntry* __restrict__ vis = reinterpret_cast<const VisEntry*>(m.visible);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int kb = (int)(t / a.n_frames), i = (int)(t - (long long)kb * a.n_frames);
        const VisEntry e = vis[kb];
        if ((e.mask >> i) & 1u)
            reinterpret_cast<VisOrigin*>(m.vis_org)[t] =
                block_origin(a, a.fr[i], reinterpret_cast<const int4*>(m.coords)[e.b]);
    }
}

// Exact float64 decision and value for voxel (i, j, k) and map `fr`, in the oracle's order.
__device__ bool fuse_voxel_f64(const float* __restrict__ depth, const FuseArgs& a, const FuseFrame& fr, int i, int j,
                               int k, float* ut) {
    double c[3];
    to_camera(fr, __dmul_rn(__dadd_rn((double)i, 0.5), a.s), __dmul_rn(__dadd_rn((double)j, 0.5), a.s),
              __dmul_rn(__dadd_rn((double)k, 0.5), a.s), c);
    if (!(c[2] > 0.0)) return false;
    const double pxf = floor(__dadd_rn(__ddiv_rn(__dmul_rn(a.fx, c[0]), c[2]), a.cx));
    const double pyf = floor(__dadd_rn(__ddiv_rn(__dmul_rn(a.fy, c[1]), c[2]), a.cy));
    if (!(pxf >= 0.0 && pxf < (double)a.W && pyf >= 0.0 && pyf < (double)a.H)) return false;
    const float d = __ldg(depth + (size_t)pyf * a.W + (size_t)pxf);
    if (!(isfinite(d) && d > 0.0f)) return false;
    const double usdf = __dsub_rn((double)d, c[2]);
    if (usdf < -a.mu) return false;
    *ut = (float)fmin(1.0, __ddiv_rn(usdf, a.mu));
    return true;
}

// floor() of a float32 projection value v with error bound e, certified when
// floor(v - e) == floor(v + e); returns false when undecided.  |v| must be below 2^21.
__device__ inline bool certified_floor(float v, float e, int* out) {
    const int lo = floor_small(v - e);
    *out = lo;
    return lo == floor_small(v + e);
}

__global__ void __launch_bounds__(128, 8) fuse_kernel(const float* __restrict__ depth, DeviceMap m, FuseArgs a) {
    __shared__ VisOrigin org[kMaxBatch];
    const int nv = m.counters[kNumVisible];
    const int t = threadIdx.x;
    const int l0 = 4 * t;
    const int lx0 = l0 & 7, ly = (l0 >> 3) & 7, lz = l0 >> 6;
    const VisEntry* __restrict__ vis = reinterpret_cast<const VisEntry*>(m.visible);
    const float lyf = (float)ly, lzf = (float)lz, lx0f = (float)lx0;
    const float eps22 = 2.38418579e-7f, eps23 = 1.19209290e-7f;  // 2^-22, 2^-23
    const float s25 = 25.0f * a.sf;
    const size_t npix = (size_t)a.W * a.H;
    // the next work-list entry is fetched one block ahead, so that a block's f, w and
    // depth loads are not queued behind the load of its own entry
    VisEntry e_next;
    if (blockIdx.x < nv) e_next = vis[blockIdx.x];
    for (int kb = blockIdx.x; kb < nv; kb += gridDim.x) {
        const VisEntry e = e_next;
        if (kb + (int)gridDim.x < nv) e_next = vis[kb + gridDim.x];
        const int b = e.b;
        // the block's origins in its maps, one thread per map
        if (t < a.n_frames && ((e.mask >> t) & 1u))
            org[t] = reinterpret_cast<const VisOrigin*>(m.vis_org)[(size_t)kb * a.n_frames + t];
        float4* fp = reinterpret_cast<float4*>(m.f + (size_t)b * kBlockVoxels) + t;
        float4* wp = reinterpret_cast<float4*>(m.w + (size_t)b * kBlockVoxels) + t;
        float4 f4 = *fp, w4 = *wp;
        float fv[4] = {f4.x, f4.y, f4.z, f4.w};
        float wv[4] = {w4.x, w4.y, w4.z, w4.w};
        bool any = false;
        __syncthreads();
        for (uint32_t mm = e.mask; mm; mm &= mm - 1u) {
            const int i = __ffs(mm) - 1;  // maps in order
            const FuseFrame& fr = a.fr[i];
            const VisOrigin vb = org[i];
            const float bex = vb.ex, bey = vb.ey;
            const float* __restrict__ dm = depth + (size_t)i * npix;
            const float dl = vb.delta;
            // local offsets along y and z are shared by the thread's four voxels
            const float myz[3] = {fmaf(fr.M[1], lyf, fr.M[2] * lzf), fmaf(fr.M[4], lyf, fr.M[5] * lzf),
                                  fmaf(fr.M[7], lyf, fr.M[8] * lzf)};
            // Decisions after the projection (px, py) of a voxel certainly in front of
            // the camera, with its error bounds: outside the image, the pixel, a valid
            // depth, u_SDF >= -mu.  Returns 1 when certified (upd, ut set), else 0.
            auto project_rest = [&](float px, float py, float ex, float ey, float mz, bool* upd, float* ut) -> int {
                int pxi, pyi;
                if (px + ex < 0.0f || px - ex >= a.Wf || py + ey < 0.0f || py - ey >= a.Hf)
                    return 1;  // the real projection is certainly outside the image
                if (!(ex < 1048576.0f && ey < 1048576.0f && certified_floor(px, ex, &pxi) &&
                      certified_floor(py, ey, &pyi)))
                    return 0;
                // certified and within (-e, W + e): the pixel lies in the image
                const float d = __ldg(dm + pyi * a.W + pxi);
                if (!(isfinite(d) && d > 0.0f)) return 1;
                // u_SDF = d - z with z = hi + mz + lo: three roundings, the error of mz, the
                // rounding of mu and of us + mu
                const float dh = d - vb.hi[2];
                const float us = (dh - mz) - vb.lo[2];
                const float eu = eps22 * (fabsf(dh) + fabsf(mz) + fabsf(us) + a.muf + s25) + dl + 1e-7f;
                if (!(fabsf(us + a.muf) > eu)) return 0;
                *upd = us >= -a.muf;
                *ut = fminf(1.0f, us * a.imuf);
                return 1;
            };
            auto update = [&](int q, bool upd, float ut) {
                if (upd) {
                    const float wn = wv[q] + 1.0f;
                    // the running mean of Eq. 1 (f is compared with a tolerance, so the fast
                    // division's two ulps do not matter; the update decision is already taken)
                    fv[q] = __fdividef(fmaf(wv[q], fv[q], ut), wn);
                    wv[q] = wn;
                    any = true;
                }
            };
            if (bex >= 0.0f) {
                // The shared bounds (the same branch for the whole CTA): every voxel of the
                // block is certainly in front (shared_projection_bound).  In phases, so
                // that the four depth reads are in flight together and the float64
                // recomputation stays off the common path: pixels, reads, u_SDF tests,
                // then the voxels left undecided.
                int pix[4];
                float mzq[4];
                unsigned need = 0u, undec = 0u;  // bit q: depth read needed / undecided
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float lx = lx0f + (float)q;
                    const float mx = fmaf(fr.M[0], lx, myz[0]);
                    const float my = fmaf(fr.M[3], lx, myz[1]);
                    const float mz = fmaf(fr.M[6], lx, myz[2]);
                    const float x = (vb.hi[0] + mx) + vb.lo[0];
                    const float y = (vb.hi[1] + my) + vb.lo[1];
                    const float z = (vb.hi[2] + mz) + vb.lo[2];
                    const float inv = rcp_approx(z);
                    const float px = fmaf(a.fxf, x * inv, a.cxf), py = fmaf(a.fyf, y * inv, a.cyf);
                    mzq[q] = mz;
                    pix[q] = 0;
                    int pxi, pyi;
                    if (px + bex < 0.0f || px - bex >= a.Wf || py + bey < 0.0f || py - bey >= a.Hf) {
                        // the real projection is certainly outside the image
                    } else if (bex < 1048576.0f && bey < 1048576.0f && certified_floor(px, bex, &pxi) &&
                               certified_floor(py, bey, &pyi)) {
                        pix[q] = pyi * a.W + pxi;  // certified and within (-e, W + e): in the image
                        need |= 1u << q;
                    } else {
                        undec |= 1u << q;
                    }
                }
                float dq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) dq[q] = ((need >> q) & 1u) ? __ldg(dm + pix[q]) : 0.0f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!((need >> q) & 1u)) continue;
                    const float d = dq[q];
                    if (!(isfinite(d) && d > 0.0f)) continue;
                    // u_SDF = d - z with z = hi + mz + lo: three roundings, the error of mz, the
                    // rounding of mu and of us + mu
                    const float dh = d - vb.hi[2];
                    const float us = (dh - mzq[q]) - vb.lo[2];
                    const float eu = eps22 * (fabsf(dh) + fabsf(mzq[q]) + fabsf(us) + a.muf + s25) + dl + 1e-7f;
                    if (fabsf(us + a.muf) > eu) update(q, us >= -a.muf, fminf(1.0f, us * a.imuf));
                    else undec |= 1u << q;
                }
                if (undec) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (!((undec >> q) & 1u)) continue;
                        float ut = 0.0f;
                        const bool upd = fuse_voxel_f64(dm, a, fr, 8 * m.coords[4 * b + 1] + lx0 + q,
                                                        8 * m.coords[4 * b + 2] + ly, 8 * m.coords[4 * b + 3] + lz, &ut);
                        update(q, upd, ut);
                    }
                }
                continue;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float lx = lx0f + (float)q;
                const float mx = fmaf(fr.M[0], lx, myz[0]);
                const float my = fmaf(fr.M[3], lx, myz[1]);
                const float mz = fmaf(fr.M[6], lx, myz[2]);
                const float x = (vb.hi[0] + mx) + vb.lo[0];
                const float y = (vb.hi[1] + my) + vb.lo[1];
                const float z = (vb.hi[2] + mz) + vb.lo[2];
                int decided = 0;  // 1: certified in float32
                bool upd = false;
                float ut = 0.0f;
                // Error of each coordinate: two roundings of |x| (the sums), the rounding
                // of M = s R^T and of its products with l <= 7 (|M l| <= 7 s sqrt(3)), the
                // origin residual; 2^-22 (|x| + 25 s) is twice 2^-24 (2 |x| + 49 s).
                const float dx = fmaf(eps22, fabsf(x) + s25, dl), dy = fmaf(eps22, fabsf(y) + s25, dl),
                            dz = fmaf(eps22, fabsf(z) + s25, dl);
                if (z + dz <= 0.0f) {
                    decided = 1;  // certainly behind the camera
                } else if (z - dz > 0.0f) {
                    const float inv = rcp_approx(z);  // z > dz > 2^-20 s: a normal number
                    const float rx = x * inv, ry = y * inv;
                    const float px = fmaf(a.fxf, rx, a.cxf);
                    const float py = fmaf(a.fyf, ry, a.cyf);
                    // |x/z - rx| <= (dx + |rx| dz) / (z - dz) from the coordinates, plus the
                    // error of the approximate 1/z (1 ulp) and the roundings of x * (1/z), the
                    // fma and of fx, cx: below 2^-24 (|px| + |cx| + 4 fx |rx|), which
                    // 2^-22 fx |rx| + 2^-23 (|px| + |cx|) covers (twice on the second part).
                    // The approximate 1/(z - dz) is within 1 ulp, which the factor 1.01 covers.
                    const float iz = rcp_approx(z - dz);
                    const float ex = a.fxf * (dx + fabsf(rx) * dz) * iz * 1.01f + eps22 * (a.fxf * fabsf(rx)) +
                                     eps23 * (fabsf(px) + fabsf(a.cxf)) + 1e-6f;
                    const float ey = a.fyf * (dy + fabsf(ry) * dz) * iz * 1.01f + eps22 * (a.fyf * fabsf(ry)) +
                                     eps23 * (fabsf(py) + fabsf(a.cyf)) + 1e-6f;
                    decided = project_rest(px, py, ex, ey, mz, &upd, &ut);
                }
                if (!decided)
                    upd = fuse_voxel_f64(dm, a, fr, 8 * m.coords[4 * b + 1] + lx0 + q, 8 * m.coords[4 * b + 2] + ly,
                                         8 * m.coords[4 * b + 3] + lz, &ut);
                update(q, upd, ut);
            }
        }
        if (any) {
            *fp = make_float4(fv[0], fv[1], fv[2], fv[3]);
            *wp = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
        __syncthreads();  // org is rewritten for the next block
    }
}

}  // namespace

int launch_fuse(denser_ctx* c, const float* depth, int n_frames, const denser_intrinsics* K, const double* T,
                int32_t segment, cudaStream_t s, bool after_alloc) {
    FuseArgs a;
    for (int i = 0; i < n_frames; ++i) {
        FuseFrame& fr = a.fr[i];
        const double* Ti = T + 16 * i;
        // inverse pose (R^T, -R^T t), each row summed left to right
        for (int r = 0; r < 3; ++r) {
            for (int q = 0; q < 3; ++q) fr.Ri[3 * r + q] = Ti[4 * q + r];
            const double v0 = Ti[4 * 0 + r] * Ti[3];
            const double v1 = Ti[4 * 1 + r] * Ti[7];
            const double v2 = Ti[4 * 2 + r] * Ti[11];
            fr.ti[r] = -((v0 + v1) + v2);
        }
        for (int e = 0; e < 9; ++e) fr.M[e] = (float)(fr.Ri[e] * c->prm.voxel_size);
        fr.tabs = 0.0f;
        for (int e = 0; e < 9; ++e) fr.Rif[e] = (float)fr.Ri[e];
        for (int e = 0; e < 3; ++e) fr.tif[e] = (float)fr.ti[e], fr.tabs += (float)fabs(fr.ti[e]);
    }
    a.n_frames = n_frames;
    a.gate = after_alloc ? 1 : 0;
    a.fx = K->fx, a.fy = K->fy, a.cx = K->cx, a.cy = K->cy;
    a.s = c->prm.voxel_size;
    a.mu = c->prm.mu;
    a.W = K->width, a.H = K->height;
    a.seg = segment;
    // side planes n.p >= 0 for points that project inside [0, W) x [0, H) (z > 0)
    const double raw[4][3] = {{K->fx, 0.0, K->cx},
                              {-K->fx, 0.0, (double)K->width - K->cx},
                              {0.0, K->fy, K->cy},
                              {0.0, -K->fy, (double)K->height - K->cy}};
    for (int q = 0; q < 4; ++q) {
        const double n = sqrt(raw[q][0] * raw[q][0] + raw[q][1] * raw[q][1] + raw[q][2] * raw[q][2]);
        for (int e = 0; e < 3; ++e) a.planef[q][e] = (float)(raw[q][e] / n);
    }
    a.radius = 3.5 * c->prm.voxel_size * sqrt(3.0) * (1.0 + 1e-9) + 1e-6;
    a.fxf = (float)a.fx, a.fyf = (float)a.fy, a.cxf = (float)a.cx, a.cyf = (float)a.cy;
    a.muf = (float)a.mu, a.sf = (float)a.s;
    a.imuf = (float)(1.0 / a.mu);
    a.Wf = (float)a.W, a.Hf = (float)a.H;
    if (!after_alloc) {
        cudaMemsetAsync(c->d.counters + kNumVisible, 0, (kCounterWords - kNumVisible) * sizeof(int32_t), s);
        const int npix = a.W * a.H;
        for (int i = 0; i < n_frames; ++i)
            depth_max_kernel<<<grid_for(c->sm_count, (npix + 3) / 4, 256, 2), 256, 0, s>>>(
                depth + (size_t)i * npix, npix, c->d.counters + kFrameDepthMax + i);
        c->launches += n_frames;
    }
    if (n_frames > c->d.org_frames) {
        // room for every map of a batch: grown once, after the queued work that reads it
        int rc = cuda_check(c, cudaStreamSynchronize(s), "stream synchronize");
        if (rc) return rc;
        cudaFree(c->d.vis_org);
        c->d.vis_org = nullptr;
        c->d.org_frames = 0;
        rc = cuda_check(c, cudaMalloc(&c->d.vis_org, (size_t)c->d.max_blocks * kMaxBatch * sizeof(VisOrigin)),
                        "cudaMalloc(fusion origins)");
        if (rc) return rc;
        c->d.org_frames = kMaxBatch;
    }
    cull_kernel<<<grid_for(c->sm_count, c->d.max_blocks, 256, 4), 256, 0, s>>>(c->d, a);
    origin_kernel<<<grid_for(c->sm_count, (int64_t)c->d.max_blocks * n_frames, 256, 8), 256, 0, s>>>(c->d, a);
    if (c->profile) cudaEventRecord(c->prof_ev[3], s);
    fuse_kernel<<<c->sm_count * 16, 128, 0, s>>>(depth, c->d, a);
    if (c->profile) cudaEventRecord(c->prof_ev[4], s);
    c->launches += 3;
    return cuda_check(c, cudaGetLastError(), "fusion kernels");
}

}  // namespace denser
