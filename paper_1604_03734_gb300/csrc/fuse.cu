// Projective TSDF fusion, Eq. 1 (Section III-A, steps 1-4).
//
// Three kernels per depth map:
//   depth_max   largest valid depth of the map (bounds the blocks that can change);
//   cull        conservative per-block test (bounding sphere of the voxel centres
//               against the camera's near plane, the viewing frustum's four side
//               planes and the far limit d_max + mu); survivors go to a work list.
//               A culled block provably has no voxel that Eq. 1 would update;
//   fuse        one CTA per listed block, 128 threads x 4 consecutive voxels; f and w
//               move as float4.  Each integer decision (the pixel a voxel projects to,
//               z_c > 0, u_SDF >= -mu) is first taken in float32 together with a
//               forward error bound; when the bound cannot certify it, the voxel is
//               recomputed in float64 in the oracle's exact operation order.  So the set
//               of updated voxels (and w) is bit-exact while float64, which runs at a
//               small fraction of the float32 rate on this GPU, is used for well under
//               1% of voxels.  f is accumulated in float32.
#include <math.h>

#include "common.cuh"

namespace denser {

namespace {

struct FuseArgs {
    double Ri[9];  // R^T
    double ti[3];  // -R^T t
    double fx, fy, cx, cy, s, mu;
    double plane[4][3];  // unit normals of the four side planes (camera frame)
    double radius;       // bounding-sphere radius of a block's voxel centres, padded
    float M[9];          // s R^T: camera-frame step per local voxel index (float32)
    float fxf, fyf, cxf, cyf, muf, sf, Wf, Hf;
    float imuf;            // 1 / mu as float32
    float Rif[9], tif[3];  // R^T and -R^T t as float32 (the culling test)
    float planef[4][3], tabs;  // side planes as float32; |t|_1 of -R^T t
    int W, H, seg;
};

// A block selected for fusion, with the camera-frame centre of its voxel (0,0,0)
// split into float32 high and low parts (hi + lo = the float64 value to ~2^-48).
struct VisBlock {
    int b;
    float hi[3];
    float lo[3];
    float delta;  // bound on |c0 - (hi + lo)| for the block
};
static_assert(sizeof(VisBlock) == 32, "VisBlock is 32 bytes");

__global__ void __launch_bounds__(256) depth_max_kernel(const float* __restrict__ depth, int n, int32_t* counters) {
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
        if (mx > 0.0f) atomicMax(counters + kDepthMaxBits, __float_as_int(mx));
    }
}

__device__ inline void to_camera(const FuseArgs& a, double gx, double gy, double gz, double* c) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        c[r] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(a.Ri[3 * r], gx), __dmul_rn(a.Ri[3 * r + 1], gy)),
                                   __dmul_rn(a.Ri[3 * r + 2], gz)),
                         a.ti[r]);
}

__global__ void cull_kernel(DeviceMap m, FuseArgs a) {
    const int nb = m.counters[kNumBlocks];
    const int dbits = m.counters[kDepthMaxBits];
    if (dbits == 0) return;  // no valid pixel: nothing can change
    const float farf = (float)((double)__int_as_float(dbits) + a.mu) * (1.0f + 1.0e-6f) + 1.0e-6f;
    const int lane = threadIdx.x & 31;
    // warp-uniform loop bound: every lane reaches the ballot
    for (int base = blockIdx.x * blockDim.x; base < nb; base += gridDim.x * blockDim.x) {
        const int b = base + (int)threadIdx.x;
        bool keep = false;
        VisBlock vb;
        if (b < nb) {
            const int4 k = reinterpret_cast<const int4*>(m.coords)[b];
            if (k.x == a.seg) {
                // centre of the block's voxel centres: voxel index 8 b + 3.5 -> (8 b + 4) s.
                // The test only skips blocks that no voxel of can be updated, so float32
                // with a margin is enough: the float32 centre and plane distances are
                // within 2^-21 (|g|_1 + |t|_1 + 1) of the exact ones, the margin is twice that.
                const float gx = (float)(8 * k.y + 4) * a.sf, gy = (float)(8 * k.z + 4) * a.sf,
                            gz = (float)(8 * k.w + 4) * a.sf;
                float c[3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    c[r] = fmaf(a.Rif[3 * r], gx, fmaf(a.Rif[3 * r + 1], gy, fmaf(a.Rif[3 * r + 2], gz, a.tif[r])));
                const float r = (float)a.radius +
                                9.53674316e-7f * (fabsf(gx) + fabsf(gy) + fabsf(gz) + a.tabs + 1.0f);
                keep = c[2] + r >= 0.0f && c[2] - r <= farf;  // not all behind, not all beyond d + mu
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    keep &= fmaf(a.planef[q][0], c[0], fmaf(a.planef[q][1], c[1], a.planef[q][2] * c[2])) >= -r;
                if (keep) {
                    double c0[3];
                    to_camera(a, __dmul_rn(__dadd_rn((double)(8 * k.y), 0.5), a.s),
                              __dmul_rn(__dadd_rn((double)(8 * k.z), 0.5), a.s),
                              __dmul_rn(__dadd_rn((double)(8 * k.w), 0.5), a.s), c0);
                    vb.b = b;
                    double amax = 0.0;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        vb.hi[e] = (float)c0[e];
                        vb.lo[e] = (float)(c0[e] - (double)vb.hi[e]);
                        amax = fmax(amax, fabs(c0[e]));
                    }
                    // What hi + lo misses of the float64 origin, and the float64 roundings of the
                    // oracle's own transform (relative 2^-51 of |R| |g| + |t| per coordinate);
                    // the float32 rounding of each voxel's coordinate is bounded per voxel in the
                    // fusion kernel.
                    const double gmax = (8.0 * (fabs((double)k.y) + fabs((double)k.z) + fabs((double)k.w)) + 24.0) * a.s;
                    const double tmax = fabs(a.ti[0]) + fabs(a.ti[1]) + fabs(a.ti[2]);
                    vb.delta = (float)(ldexp(amax + gmax + tmax + 1.0, -44));
                }
            }
        }
        // one atomic per warp for the work-list slots
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        int first = 0;
        if (lane == 0 && ball) first = atomicAdd(m.counters + kNumVisible, __popc(ball));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (keep) reinterpret_cast<VisBlock*>(m.visible)[first + __popc(ball & ((1u << lane) - 1))] = vb;
    }
}

// Exact float64 decision and value for voxel (i, j, k), in the oracle's order.
__device__ bool fuse_voxel_f64(const float* __restrict__ depth, const FuseArgs& a, int i, int j, int k, float* ut) {
    double c[3];
    to_camera(a, __dmul_rn(__dadd_rn((double)i, 0.5), a.s), __dmul_rn(__dadd_rn((double)j, 0.5), a.s),
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
    const int nv = m.counters[kNumVisible];
    const int t = threadIdx.x;
    const int l0 = 4 * t;
    const int lx0 = l0 & 7, ly = (l0 >> 3) & 7, lz = l0 >> 6;
    const VisBlock* __restrict__ vis = reinterpret_cast<const VisBlock*>(m.visible);
    const float lyf = (float)ly, lzf = (float)lz, lx0f = (float)lx0;
    const float eps22 = 2.38418579e-7f;  // 2^-22
    const float s25 = 25.0f * a.sf;
    // the next work-list entry is fetched one block ahead, so that a block's f, w and
    // depth loads are not queued behind the load of its own entry
    VisBlock vb_next;
    if (blockIdx.x < nv) vb_next = vis[blockIdx.x];
    for (int kb = blockIdx.x; kb < nv; kb += gridDim.x) {
        const VisBlock vb = vb_next;
        if (kb + (int)gridDim.x < nv) vb_next = vis[kb + gridDim.x];
        const int b = vb.b;
        float4* fp = reinterpret_cast<float4*>(m.f + (size_t)b * kBlockVoxels) + t;
        float4* wp = reinterpret_cast<float4*>(m.w + (size_t)b * kBlockVoxels) + t;
        float4 f4 = *fp, w4 = *wp;
        float fv[4] = {f4.x, f4.y, f4.z, f4.w};
        float wv[4] = {w4.x, w4.y, w4.z, w4.w};
        bool any = false;
        const float dl = vb.delta;
        // local offsets along y and z are shared by the thread's four voxels
        const float myz[3] = {fmaf(a.M[1], lyf, a.M[2] * lzf), fmaf(a.M[4], lyf, a.M[5] * lzf),
                              fmaf(a.M[7], lyf, a.M[8] * lzf)};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float lx = lx0f + (float)q;
            const float mx = fmaf(a.M[0], lx, myz[0]);
            const float my = fmaf(a.M[3], lx, myz[1]);
            const float mz = fmaf(a.M[6], lx, myz[2]);
            const float x = (vb.hi[0] + mx) + vb.lo[0];
            const float y = (vb.hi[1] + my) + vb.lo[1];
            const float z = (vb.hi[2] + mz) + vb.lo[2];
            // Error of each coordinate: two roundings of |x| (the sums), the rounding of
            // M = s R^T and of its products with l <= 7 (|M l| <= 7 s sqrt(3)), the origin
            // residual; 2^-22 (|x| + 25 s) is twice 2^-24 (2 |x| + 49 s).
            const float dx = fmaf(eps22, fabsf(x) + s25, dl), dy = fmaf(eps22, fabsf(y) + s25, dl),
                        dz = fmaf(eps22, fabsf(z) + s25, dl);
            int decided = 0;  // 1: certified in float32
            bool upd = false;
            float ut = 0.0f;
            if (z + dz <= 0.0f) {
                decided = 1;  // certainly behind the camera
            } else if (z - dz > 0.0f) {
                const float inv = __frcp_rn(z);
                const float rx = x * inv, ry = y * inv;
                const float px = fmaf(a.fxf, rx, a.cxf);
                const float py = fmaf(a.fyf, ry, a.cyf);
                // |x/z - rx| <= (dx + |rx| dz) / (z - dz) from the coordinates, plus the
                // roundings of 1/z, x * (1/z), the fma and of fx, cx (below 2^-24 (|px| + |cx| +
                // 3 fx |rx|)); 2^-22 (fx |rx| + |px| + |cx|) covers those with margin.
                const float iz = __frcp_rn(z - dz);
                const float ex = a.fxf * (dx + fabsf(rx) * dz) * iz * 1.01f + eps22 * (a.fxf * fabsf(rx) + fabsf(px) + fabsf(a.cxf)) + 1e-6f;
                const float ey = a.fyf * (dy + fabsf(ry) * dz) * iz * 1.01f + eps22 * (a.fyf * fabsf(ry) + fabsf(py) + fabsf(a.cyf)) + 1e-6f;
                int pxi, pyi;
                if (px + ex < 0.0f || px - ex >= a.Wf || py + ey < 0.0f || py - ey >= a.Hf) {
                    decided = 1;  // the real projection is certainly outside the image
                } else if (ex < 1048576.0f && ey < 1048576.0f && certified_floor(px, ex, &pxi) &&
                           certified_floor(py, ey, &pyi)) {
                    // certified and within (-e, W + e): the pixel lies in the image
                    const float d = __ldg(depth + pyi * a.W + pxi);
                    if (!(isfinite(d) && d > 0.0f)) {
                        decided = 1;
                    } else {
                        // u_SDF = d - z with z = hi + mz + lo: three roundings, the error of mz,
                        // the rounding of mu and of us + mu
                        const float dh = d - vb.hi[2];
                        const float us = (dh - mz) - vb.lo[2];
                        const float eu = eps22 * (fabsf(dh) + fabsf(mz) + fabsf(us) + a.muf + s25) + dl + 1e-7f;
                        if (fabsf(us + a.muf) > eu) {
                            decided = 1;
                            upd = us >= -a.muf;
                            ut = fminf(1.0f, us * a.imuf);
                        }
                    }
                }
            }
            if (!decided) upd = fuse_voxel_f64(depth, a, 8 * m.coords[4 * b + 1] + lx0 + q, 8 * m.coords[4 * b + 2] + ly,
                                               8 * m.coords[4 * b + 3] + lz, &ut);
            if (upd) {
                const float wn = wv[q] + 1.0f;
                // the running mean of Eq. 1 (f is compared with a tolerance, so the fast
                // division's two ulps do not matter; the update decision is already taken)
                fv[q] = __fdividef(fmaf(wv[q], fv[q], ut), wn);
                wv[q] = wn;
                any = true;
            }
        }
        if (any) {
            *fp = make_float4(fv[0], fv[1], fv[2], fv[3]);
            *wp = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
    }
}

}  // namespace

int launch_fuse(denser_ctx* c, const float* depth, const denser_intrinsics* K, const double* T, int32_t segment,
                cudaStream_t s, bool depth_max_ready) {
    FuseArgs a;
    // inverse pose (R^T, -R^T t), each row summed left to right
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) a.Ri[3 * r + q] = T[4 * q + r];
        const double v0 = T[4 * 0 + r] * T[3];
        const double v1 = T[4 * 1 + r] * T[7];
        const double v2 = T[4 * 2 + r] * T[11];
        a.ti[r] = -((v0 + v1) + v2);
    }
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
        for (int e = 0; e < 3; ++e) a.plane[q][e] = raw[q][e] / n;
    }
    a.radius = 3.5 * c->prm.voxel_size * sqrt(3.0) * (1.0 + 1e-9) + 1e-6;
    for (int e = 0; e < 9; ++e) a.M[e] = (float)(a.Ri[e] * a.s);
    a.fxf = (float)a.fx, a.fyf = (float)a.fy, a.cxf = (float)a.cx, a.cyf = (float)a.cy;
    a.muf = (float)a.mu, a.sf = (float)a.s;
    a.imuf = (float)(1.0 / a.mu);
    a.Wf = (float)a.W, a.Hf = (float)a.H;
    a.tabs = 0.0f;
    for (int e = 0; e < 9; ++e) a.Rif[e] = (float)a.Ri[e];
    for (int e = 0; e < 3; ++e) a.tif[e] = (float)a.ti[e], a.tabs += (float)fabs(a.ti[e]);
    for (int q = 0; q < 4; ++q)
        for (int e = 0; e < 3; ++e) a.planef[q][e] = (float)a.plane[q][e];
    if (!depth_max_ready) {
        cudaMemsetAsync(c->d.counters + kNumVisible, 0, 2 * sizeof(int32_t), s);
        const int npix = a.W * a.H;
        depth_max_kernel<<<grid_for(c->sm_count, (npix + 3) / 4, 256, 2), 256, 0, s>>>(depth, npix, c->d.counters);
        c->launches += 1;
    }
    cull_kernel<<<grid_for(c->sm_count, c->d.max_blocks, 256, 4), 256, 0, s>>>(c->d, a);
    fuse_kernel<<<c->sm_count * 16, 128, 0, s>>>(depth, c->d, a);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "fusion kernels");
}

}  // namespace denser
