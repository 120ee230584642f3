// Laser ray fusion (Section III-A: the projective update extends to laser sensors by
// updating only the voxels along each ray, from the sensor to mu behind the observed
// surface).  Readings, also stated with the oracle:
//   * the voxels along a ray are those holding a ray sample at range n h, n = 0..M,
//     M = floor((r + mu) / h), h = s/2, in an allocated block of the scan's segment; a
//     voxel counts once per ray; a point with M >= 2^22 (beyond about 200 km at 10 cm
//     voxels) is not valid;
//   * such a voxel (centre c) observes u_SDF = r - (c - t) . dg, taken when
//     u_SDF >= -mu, as u_TSDF = min(1, u_SDF / mu);
//   * a scan updates a voxel once with all its observations, w += n and
//     f = (w f + sum u_TSDF) / w, the sum in fixed point (multiples of 2^-30), so that
//     the result does not depend on the order in which rays land.
//
// Two kernels.  march: one thread per point walks the ray's samples in float32,
// certified against one error bound per ray and axis (float64 in the oracle's order
// when a floor or the truncation test is too close to call), looks blocks up only when
// the sample's block changes, jumps over the samples of unallocated blocks, and adds
// (1 << 48) + round(u_TSDF 2^30) to the voxel's 64-bit accumulator.  finalize: one CTA
// per touched block folds the accumulators into f and w (float64 arithmetic, float32
// storage) and clears them.
#include "common.cuh"

namespace denser {

namespace {

constexpr double kFix = 1073741824.0;  // 2^30
constexpr unsigned long long kCountOne = 1ull << 48;

struct MarchArgs {
    double R[9], t[3];
    double s, h, mu;
    int Tv[3];     // floor(t / s)
    float tf[3];   // t / s - Tv, in [0, 1)
    double tfd[3]; // the same in float64
    float sf, muf;
    int seg;
    long long n;   // points
};

__device__ __forceinline__ int floor_rel(float q, float e, bool* ok) {
    // floor(q) by a round-to-nearest add (|q| < 2^22), certified when q stays e away
    // from both neighbouring integers
    const float tq = __fadd_rn(q, 12582912.0f);
    const float nq = tq - 12582912.0f;
    const bool down = nq > q;
    const float fr = q - (down ? nq - 1.0f : nq);
    *ok = *ok && fr >= e && 1.0f - fr > e;
    return __float_as_int(tq) - 0x4B400000 - (down ? 1 : 0);
}

__global__ void __launch_bounds__(128) laser_march_kernel(const float* __restrict__ pts, MarchArgs a, DeviceMap m,
                                                          unsigned long long* __restrict__ acc,
                                                          uint8_t* __restrict__ touched) {
    const float eps19 = 1.90734863e-6f, eps20 = 9.53674316e-7f, eps22 = 2.38418579e-7f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
         i += (long long)gridDim.x * blockDim.x) {
        double r, dg[3];
        if (!laser_ray(a.R, __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2), &r, dg)) continue;
        const double Md = floor(__ddiv_rn(__dadd_rn(r, a.mu), a.h));
        if (!(Md < 4194304.0)) continue;  // range beyond 2^22 samples: not a valid point
        const int M = (int)Md;
        // q = t/s + n (h/s) dg relative to Tv, h/s = 1/2 exactly, with the step held as a
        // float32 pair Dh + Dl: q = fma(n, Dh, fma(n, Dl, tf)).  Per-axis bound
        //   |q - q_real| <= 2^-24 (|q| + 2) + 2^-48 n |Dh|  (the two fmas, tf, the pair),
        //   e = 2^-22 (M |Dh| + 3) covers it at least 4 times.
        float Dh[3], Dl[3], e[3], Dg[3];
        bool fast = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Dg[k] = (float)dg[k];
            const double half = 0.5 * dg[k];
            Dh[k] = (float)half;
            Dl[k] = (float)(half - (double)Dh[k]);
            const float span = (float)M * fabsf(Dh[k]);
            fast = fast && span < 2097152.0f;
            e[k] = eps22 * (span + 3.0f);
        }
        // the hit point in voxel units relative to Tv, P = r dg / s + (t / s - Tv), as a
        // float32 pair hi + lo: the signed distance of a voxel is then a short vector
        // product, u_SDF = -s (c/s - Tv - P) . dg, without the cancellation of r - (c - t) . dg
        float Phi[3], Plo[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double P = __dadd_rn(__ddiv_rn(__dmul_rn(r, dg[k]), a.s), a.tfd[k]);
            Phi[k] = (float)P;
            Plo[k] = (float)(P - (double)Phi[k]);
        }
        int last0 = INT_MIN, last1 = 0, last2 = 0;  // last voxel (relative to Tv)
        int lb0 = INT_MIN, lb1 = 0, lb2 = 0, lidx = -1;  // last block looked up and its index
        float nf = 0.0f;
        for (int n = 0; n <= M; ++n, nf += 1.0f) {
            int k0, k1, k2;
            bool ok = fast;
            if (ok) {
                k0 = floor_rel(fmaf(nf, Dh[0], fmaf(nf, Dl[0], a.tf[0])), e[0], &ok);
                k1 = floor_rel(fmaf(nf, Dh[1], fmaf(nf, Dl[1], a.tf[1])), e[1], &ok);
                k2 = floor_rel(fmaf(nf, Dh[2], fmaf(nf, Dl[2], a.tf[2])), e[2], &ok);
            }
            if (!ok) {
                const double rho = __dmul_rn((double)n, a.h);
                double v[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) v[k] = floor(__ddiv_rn(__dadd_rn(__dmul_rn(dg[k], rho), a.t[k]), a.s));
                if (!(fabs(v[0]) < 2097152.0 && fabs(v[1]) < 2097152.0 && fabs(v[2]) < 2097152.0)) continue;
                k0 = (int)v[0] - a.Tv[0], k1 = (int)v[1] - a.Tv[1], k2 = (int)v[2] - a.Tv[2];
            }
            if (k0 == last0 && k1 == last1 && k2 == last2) continue;  // the same voxel as before
            last0 = k0, last1 = k1, last2 = k2;
            const int V0 = a.Tv[0] + k0, V1 = a.Tv[1] + k1, V2 = a.Tv[2] + k2;
            const int B0 = V0 >> 3, B1 = V1 >> 3, B2 = V2 >> 3;  // floor division by 8
            if (B0 != lb0 || B1 != lb1 || B2 != lb2) {
                lb0 = B0, lb1 = B1, lb2 = B2;
                lidx = key_in_range(a.seg, B0, B1, B2) ? hash_lookup(m, pack_key(a.seg, B0, B1, B2)) : -1;
            }
            if (lidx < 0) {
                // an unallocated block: jump to one sample before the first that may
                // leave it (the floors stay 2 e inside its faces until then)
                if (fast) {
                    // sample n' stays inside along axis k while tf + n' Dh is more than mq
                    // from the face: mq covers twice the floor bound and twice the rounding
                    // of the numerator below; the quotient's own rounding (2^-24 relative)
                    // is covered by stopping two samples short
                    float nx = 3.0e38f;
                    const int lo[3] = {8 * B0 - a.Tv[0], 8 * B1 - a.Tv[1], 8 * B2 - a.Tv[2]};
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float mq = 2.0f * e[k] + 2.38418579e-7f * (fabsf((float)lo[k]) + 9.0f);
                        if (Dh[k] > 0.0f) nx = fminf(nx, (((float)(lo[k] + 8) - a.tf[k]) - mq) / Dh[k]);
                        else if (Dh[k] < 0.0f) nx = fminf(nx, (((float)lo[k] - a.tf[k]) + mq) / Dh[k]);
                    }
                    // next sample to look at: jump (> n + 1), or past the end when the rest
                    // of the ray stays in the block; either way n strictly grows
                    const float jump = floorf(nx) - 2.0f;
                    if (jump > (float)n + 1.0f) {
                        const int nn = jump >= (float)M ? M + 1 : (int)jump;
                        n = nn - 1;
                        nf = (float)nn - 1.0f;
                    }
                }
                continue;
            }
            // u_SDF = r - (c - t) . dg = -s (k + 1/2 - P) . dg (dg a unit vector)
            const float q0 = ((float)k0 + 0.5f - Phi[0]) - Plo[0];
            const float q1 = ((float)k1 + 0.5f - Phi[1]) - Plo[1];
            const float q2 = ((float)k2 + 0.5f - Phi[2]) - Plo[2];
            const float dq = fabsf(q0) + fabsf(q1) + fabsf(q2);
            float u = -fmaf(q2, Dg[2], fmaf(q1, Dg[1], q0 * Dg[0])) * a.sf;
            // |u - u_real| <= s 2^-21 (|q0| + |q1| + |q2|) + 2^-22 |u| + 10^-11 s (the
            // roundings of q, Dg, the products, s; P to 2^-48); the bound below is four
            // times that, plus the rounding of mu and of u + mu
            const float eu = fmaf(eps19 * a.sf, dq + 1.0e-4f, eps20 * (fabsf(u) + a.muf));
            bool upd;
            if (fabsf(u + a.muf) > eu) {
                upd = u >= -a.muf;
            } else {
                double ed[3];
                const int V[3] = {V0, V1, V2};
#pragma unroll
                for (int k = 0; k < 3; ++k) ed[k] = __dsub_rn(__dmul_rn(__dadd_rn((double)V[k], 0.5), a.s), a.t[k]);
                const double ud = __dsub_rn(r, __dadd_rn(__dadd_rn(__dmul_rn(ed[0], dg[0]), __dmul_rn(ed[1], dg[1])),
                                                         __dmul_rn(ed[2], dg[2])));
                upd = ud >= -a.mu;
                u = (float)ud;
            }
            if (!upd) continue;
            const float ut = fminf(1.0f, u / a.muf);
            const long long q = (long long)__float2int_rn(ut * 1073741824.0f);
            const size_t v = (size_t)lidx * kBlockVoxels + (size_t)((V0 & 7) + 8 * (V1 & 7) + 64 * (V2 & 7));
            atomicAdd(acc + v, kCountOne + (unsigned long long)q);
            touched[lidx] = 1;
        }
    }
}

__global__ void __launch_bounds__(128) laser_finalize_kernel(DeviceMap m, unsigned long long* __restrict__ acc,
                                                             uint8_t* __restrict__ touched) {
    const int nb = m.counters[kNumBlocks];
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        if (!touched[b]) continue;  // uniform across the CTA
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const size_t v = (size_t)b * kBlockVoxels + threadIdx.x + 128 * q;
            const long long P = (long long)acc[v];
            if (P == 0) continue;
            // P = n 2^48 + S with |S| < 2^47: n = round(P / 2^48)
            const long long cnt = (P + (1ll << 47)) >> 48;
            const long long S = P - (cnt << 48);
            const double w0 = m.w[v];
            const double wn = w0 + (double)cnt;
            m.f[v] = (float)((w0 * (double)m.f[v] + (double)S / kFix) / wn);
            m.w[v] = (float)wn;
            acc[v] = 0ull;
        }
        __syncthreads();
        if (threadIdx.x == 0) touched[b] = 0;
    }
}

}  // namespace

int launch_fuse_points(denser_ctx* c, const float* pts, int64_t n, const double* T, int32_t segment,
                       cudaStream_t s) {
    if (!c->laser_acc) {
        int rc = cuda_check(c, cudaMalloc(&c->laser_acc, (size_t)c->d.max_blocks * kBlockVoxels * 8),
                            "cudaMalloc(laser accumulators)");
        if (rc) return rc;
        rc = cuda_check(c, cudaMalloc(&c->laser_touched, c->d.max_blocks), "cudaMalloc(laser flags)");
        if (rc) return rc;
        rc = cuda_check(c, cudaMemsetAsync(c->laser_acc, 0, (size_t)c->d.max_blocks * kBlockVoxels * 8, s),
                        "clear laser accumulators");
        if (rc) return rc;
        rc = cuda_check(c, cudaMemsetAsync(c->laser_touched, 0, c->d.max_blocks, s), "clear laser flags");
        if (rc) return rc;
    }
    if (n <= 0) return DENSER_OK;
    MarchArgs a;
    a.s = c->prm.voxel_size;
    a.h = 0.5 * a.s;
    a.mu = c->prm.mu;
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) a.R[3 * r + q] = T[4 * r + q];
        a.t[r] = T[4 * r + 3];
        const double tv = a.t[r] / a.s;
        const double ti = floor(tv);
        a.Tv[r] = (int)std::max(-8.0 * kCoordBias, std::min(8.0 * kCoordBias, ti));
        a.tfd[r] = tv - (double)a.Tv[r];
        a.tf[r] = (float)a.tfd[r];
    }
    a.sf = (float)a.s;
    a.muf = (float)a.mu;
    a.seg = segment;
    a.n = n;
    laser_march_kernel<<<grid_for(c->sm_count, n, 128, 16), 128, 0, s>>>(pts, a, c->d, c->laser_acc,
                                                                         c->laser_touched);
    laser_finalize_kernel<<<c->sm_count * 8, 128, 0, s>>>(c->d, c->laser_acc, c->laser_touched);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "laser fusion kernels");
}

}  // namespace denser
