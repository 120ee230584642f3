// Projective TSDF fusion, Eq. 1 (Section III-A, steps 1-4).
//
// Three kernels per depth map:
//   depth_max   largest valid depth of the map (bounds the blocks that can change);
//   cull        conservative per-block test (bounding sphere of the voxel centres
//               against the camera's near plane, the viewing frustum's four side
//               planes and the far limit d_max + mu); survivors go to a work list.
//               A culled block provably has no voxel that Eq. 1 would update;
//   fuse        one CTA per listed block, 128 threads x 4 consecutive voxels; f and w
//               move as float4.  The projection and the update test run in float64 in
//               the oracle's operation order, so the set of updated voxels (and so w)
//               is bit-exact; f is accumulated in float32.
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
    int W, H, seg;
};

__global__ void depth_max_kernel(const float* __restrict__ depth, int n, int32_t* counters) {
    float mx = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float d = __ldg(depth + i);
        if (isfinite(d) && d > mx) mx = d;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0f) atomicMax(counters + kDepthMaxBits, __float_as_int(mx));
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
    const double far = (double)__int_as_float(dbits) + a.mu;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int4 k = reinterpret_cast<const int4*>(m.coords)[b];
        if (k.x != a.seg) continue;
        // centre of the block's voxel centres: voxel index 8 b + 3.5 -> (8 b + 4) s
        double c[3];
        to_camera(a, (8.0 * k.y + 4.0) * a.s, (8.0 * k.z + 4.0) * a.s, (8.0 * k.w + 4.0) * a.s, c);
        const double r = a.radius;
        if (c[2] + r < 0.0) continue;    // every voxel behind the camera
        if (c[2] - r > far) continue;    // every voxel beyond any depth + mu
        bool out = false;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            out |= a.plane[q][0] * c[0] + a.plane[q][1] * c[1] + a.plane[q][2] * c[2] < -r;
        if (out) continue;
        const int pos = atomicAdd(m.counters + kNumVisible, 1);
        m.visible[pos] = b;
    }
}

__global__ void __launch_bounds__(128) fuse_kernel(const float* __restrict__ depth, DeviceMap m, FuseArgs a) {
    const int nv = m.counters[kNumVisible];
    const int t = threadIdx.x;
    const int l0 = 4 * t;
    const int lx0 = l0 & 7, ly = (l0 >> 3) & 7, lz = l0 >> 6;
    for (int k = blockIdx.x; k < nv; k += gridDim.x) {
        const int b = m.visible[k];
        const int4 key = reinterpret_cast<const int4*>(m.coords)[b];
        float4* fp = reinterpret_cast<float4*>(m.f + (size_t)b * kBlockVoxels) + t;
        float4* wp = reinterpret_cast<float4*>(m.w + (size_t)b * kBlockVoxels) + t;
        float4 f4 = *fp, w4 = *wp;
        float fv[4] = {f4.x, f4.y, f4.z, f4.w};
        float wv[4] = {w4.x, w4.y, w4.z, w4.w};
        bool any = false;
        const double gy = __dmul_rn(__dadd_rn((double)(8 * key.z + ly), 0.5), a.s);
        const double gz = __dmul_rn(__dadd_rn((double)(8 * key.w + lz), 0.5), a.s);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double gx = __dmul_rn(__dadd_rn((double)(8 * key.y + lx0 + q), 0.5), a.s);
            double c[3];
            to_camera(a, gx, gy, gz, c);
            if (!(c[2] > 0.0)) continue;
            const double pxf = floor(__dadd_rn(__ddiv_rn(__dmul_rn(a.fx, c[0]), c[2]), a.cx));
            const double pyf = floor(__dadd_rn(__ddiv_rn(__dmul_rn(a.fy, c[1]), c[2]), a.cy));
            if (!(pxf >= 0.0 && pxf < (double)a.W && pyf >= 0.0 && pyf < (double)a.H)) continue;
            const float d = __ldg(depth + (size_t)pyf * a.W + (size_t)pxf);
            if (!(isfinite(d) && d > 0.0f)) continue;
            const double usdf = __dsub_rn((double)d, c[2]);
            if (usdf < -a.mu) continue;
            const float ut = (float)fmin(1.0, __ddiv_rn(usdf, a.mu));
            const float wn = wv[q] + 1.0f;
            fv[q] = (ut + wv[q] * fv[q]) / wn;
            wv[q] = wn;
            any = true;
        }
        if (any) {
            *fp = make_float4(fv[0], fv[1], fv[2], fv[3]);
            *wp = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
    }
}

}  // namespace

int launch_fuse(denser_ctx* c, const float* depth, const denser_intrinsics* K, const double* T, int32_t segment,
                cudaStream_t s) {
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
    cudaMemsetAsync(c->d.counters + kNumVisible, 0, 2 * sizeof(int32_t), s);
    const int npix = a.W * a.H;
    depth_max_kernel<<<grid_for(c->sm_count, npix, 256, 4), 256, 0, s>>>(depth, npix, c->d.counters);
    cull_kernel<<<grid_for(c->sm_count, c->d.max_blocks, 256, 4), 256, 0, s>>>(c->d, a);
    fuse_kernel<<<c->sm_count * 16, 128, 0, s>>>(depth, c->d, a);
    c->launches += 3;
    return cuda_check(c, cudaGetLastError(), "fusion kernels");
}

}  // namespace denser
