// Block allocation into the hashing voxel grid (Section III-A, "Fusing Data").
//
// One allocation call (one depth map, or a batch of up to kMaxBatch maps of one camera)
// runs five kernels on the caller's stream, with every count kept on the device (no
// host round trip):
//   alloc_keys    one thread per pixel of every map; the band samples of the pixel's ray
//                 give block keys (certified float32, else float64 in a fixed operation
//                 order); warp peers with the same key elect one leader (match.any) that
//                 inserts it by CAS into the open-addressing table, appends it to the
//                 call's new-key list when it is new, and lowers the slot's birth (the
//                 first map of the batch that reached the key) by an atomic min;
//   sort_chunks   bitonic sort of the new keys by (birth, key), kNewKeyChunk keys per CTA
//                 in shared memory;
//   rank_assign   global rank of each new key = its rank in its chunk plus a binary
//                 search in every other chunk; block index = blocks so far + rank, which
//                 makes indices independent of insertion order and equal to those of one
//                 call per map (that order is by map, then by key);
//   pool_init     zero the new blocks' fields;
//   commit        publish the new block count.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace denser {

namespace {

// The pose of one depth map of the call.
struct AllocFrame {
    double R[9];
    double t[3];
    int Ti[3];             // floor(t / bs)
    float tf[3];           // t / bs - Ti, in [0, 1)
    float Rf[9];           // R as float32
};

struct AllocArgs {
    double fx, fy, cx, cy;
    double h;   // sample spacing s/2
    double bs;  // block size 8 s
    float hf;              // h as float32
    float cx_hi, cx_lo, cy_hi, cy_lo;  // principal point as float32 hi + lo
    float nhf;             // N h as float32
    unsigned long long w_magic;  // ceil(2^64 / W): y = umulhi(pixel, w_magic) for pixel < 2^32
    float ifx, ify, ibs;   // 1/fx, 1/fy, 1/bs as float32
    int W, H, N, seg;
    int n_frames;          // depth maps of the call, [n_frames][H][W] back to back
    int tiles;             // 256-pixel tiles per map
    AllocFrame fr[kMaxBatch];
};

constexpr unsigned long long kCoordMask = (1ull << (3 * kCoordBits)) - 1;  // a key without its segment
constexpr int kBirthShift = 3 * kCoordBits;

__device__ inline void report(int32_t* counters, int32_t bit) { atomicOr(counters + kErrorBits, bit); }

// Inserts `key`, reached by depth map `frame` of the call; returns true if this call
// created it.
__device__ bool hash_insert(const DeviceMap& m, unsigned long long key, int frame) {
    const uint32_t h = hash_key(key);
    for (int i = 0; i < kMaxProbe; ++i) {
        const uint32_t slot = (h + (uint32_t)i) & m.slot_mask;
        unsigned long long cur = __ldcg(m.hash_keys + slot);
        if (cur == key) {
            atomicMin(m.hash_birth + slot, frame);
            return false;
        }
        if (cur == kEmptyKey) {
            cur = atomicCAS(m.hash_keys + slot, kEmptyKey, key);
            if (cur == kEmptyKey) {
                atomicMin(m.hash_birth + slot, frame);
                const int pos = atomicAdd(m.counters + kNumNew, 1);
                if (pos < (int)m.max_new) {
                    m.new_keys[pos] = key;
                    m.new_slots[pos] = slot;
                } else {
                    report(m.counters, kErrNewFull);
                }
                return true;
            }
            if (cur == key) {
                atomicMin(m.hash_birth + slot, frame);
                return false;
            }
        }
    }
    report(m.counters, kErrHashFull);
    return false;
}

// Block key of band sample n of pixel (x, y) with depth d, or kEmptyKey when z <= 0.
// The float64 operations follow the oracle's order one by one; the _rn intrinsics keep
// the compiler from contracting them into fused multiply-adds.
__device__ __forceinline__ unsigned long long sample_key(const AllocArgs& a, const AllocFrame& fr, int x, int y, double d,
                                                        int n, bool* range_err) {
    const double z = __dadd_rn(d, __dmul_rn((double)n, a.h));
    if (!(z > 0.0)) return kEmptyKey;
    const double uu = __dsub_rn(__dadd_rn((double)x, 0.5), a.cx);
    const double vv = __dsub_rn(__dadd_rn((double)y, 0.5), a.cy);
    const double X = __ddiv_rn(__dmul_rn(uu, z), a.fx);
    const double Y = __ddiv_rn(__dmul_rn(vv, z), a.fy);
    const double Z = z;
    double k[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double g = __dadd_rn(
            __dadd_rn(__dadd_rn(__dmul_rn(fr.R[3 * r + 0], X), __dmul_rn(fr.R[3 * r + 1], Y)), __dmul_rn(fr.R[3 * r + 2], Z)),
            fr.t[r]);
        k[r] = floor(__ddiv_rn(g, a.bs));
    }
    if (!(k[0] >= -kCoordBias && k[0] < kCoordBias && k[1] >= -kCoordBias && k[1] < kCoordBias &&
          k[2] >= -kCoordBias && k[2] < kCoordBias)) {
        *range_err = true;
        return kEmptyKey;
    }
    return pack_key(a.seg, (int32_t)k[0], (int32_t)k[1], (int32_t)k[2]);
}

// A ray's distinct keys, held in four registers (selected by constant indices only, so
// that they never spill to local memory).
struct RayKeys {
    unsigned long long k0 = kEmptyKey, k1 = kEmptyKey, k2 = kEmptyKey, k3 = kEmptyKey;
    int count = 0;
    __device__ void push(unsigned long long k) {
        if (count == 0) k0 = k;
        else if (count == 1) k1 = k;
        else if (count == 2) k2 = k;
        else k3 = k;
        ++count;
    }
    __device__ unsigned long long at(int i) const {
        return i == 0 ? k0 : (i == 1 ? k1 : (i == 2 ? k2 : (i == 3 ? k3 : kEmptyKey)));
    }
};

// Inserts the pending keys of a warp: round after round every lane offers its next key,
// lanes offering the same key elect one leader (match.any), and the leaders insert.
__device__ inline void warp_insert(const DeviceMap& m, const RayKeys& rk, int lane, int frame) {
    for (int i = 0;; ++i) {
        const unsigned long long key = i < rk.count ? rk.at(i) : kEmptyKey;
        const unsigned active = __ballot_sync(0xffffffffu, key != kEmptyKey);
        if (!active) break;
        if (key != kEmptyKey) {
            const unsigned peers = __match_any_sync(active, key);
            if (lane == __ffs(peers) - 1) hash_insert(m, key, frame);
        }
    }
}

// Certified floor of axis coordinate q = fma(z, D, tf) of band sample nf (z = fma(nf, h,
// d), exactly as the per-sample path evaluates it); *ok is cleared when the bound e does
// not decide the floor.
__device__ __forceinline__ int band_floor(float dv, float nf, float hf, float D, float tf, float e, bool* ok) {
    const float q = fmaf(fmaf(nf, hf, dv), D, tf);
    const float tq = __fadd_rn(q, 12582912.0f);  // nearest integer + 1.5 2^23
    const float nq = tq - 12582912.0f;
    const bool down = nq > q;
    const float fr = q - (down ? nq - 1.0f : nq);  // q - floor(q), exact
    *ok = *ok && fr >= e && 1.0f - fr > e;
    return __float_as_int(tq) - 0x4B400000 - (down ? 1 : 0);
}

__device__ __forceinline__ void push_key(const DeviceMap& m, RayKeys& rk, unsigned long long key, int frame) {
    if (rk.count == 4) {  // more keys than registers: insert what is held (divergent, rare)
        hash_insert(m, rk.k0, frame), hash_insert(m, rk.k1, frame), hash_insert(m, rk.k2, frame),
            hash_insert(m, rk.k3, frame);
        rk.count = 0;
    }
    rk.push(key);
}

// The distinct block keys of a ray's band without visiting every sample.  The real
// coordinate q is linear in the sample index n, so each axis's floors are monotone along
// the band: the floors at both ends, and for each axis that changes the first sample of
// each new floor (estimated from the line, then confirmed by certified comparisons of q
// with the new floor's boundary on both sides), give every key in sample order.
// Returns false, having pushed nothing, when a decision is not certified, the nearest
// sample is not certainly in front of the camera, or an axis changes more than twice;
// the per-sample path then takes the ray.  Everything stays in registers: per axis the
// samples of at most two floor changes, merged in sample order at the end.
__device__ bool band_keys_by_events(const AllocArgs& a, const AllocFrame& fr, int frame, float dv, const float* D,
                                    const float* e, float ez, const DeviceMap& m, RayKeys& rk, bool* range_err) {
    constexpr int kNone = INT_MAX;
    const int N = a.N;
    if (!(fmaf((float)(-N), a.hf, dv) > ez)) return false;
    bool ok = true;
    int klo[3], khi[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        klo[r] = band_floor(dv, (float)(-N), a.hf, D[r], fr.tf[r], e[r], &ok);
        khi[r] = band_floor(dv, (float)N, a.hf, D[r], fr.tf[r], e[r], &ok);
    }
    if (!ok) return false;
    int n1[3], n2[3], st[3];  // per axis: the samples of its first and second floor change
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        n1[r] = kNone, n2[r] = kNone, st[r] = 0;
        const int span = khi[r] - klo[r];
        if (span == 0) continue;
        const float slope = a.hf * D[r];
        // consecutive samples move q by less than 1/2, so the floor takes every value
        // between its ends and changes at most once between two samples
        if (span > 2 || span < -2 || !(fabsf(slope) < 0.5f)) return false;
        const int step = span > 0 ? 1 : -1;
        st[r] = step;
        const float q0 = fmaf(dv, D[r], fr.tf[r]);
        for (int j = 1; j <= span * step; ++j) {
            const int v = klo[r] + j * step;
            // increasing: the first n with q >= v; decreasing: the first n with q < v + 1
            // (an estimate only, confirmed below, so the fast approximate division serves)
            const float T = step > 0 ? (float)v : (float)(v + 1);
            const float est = __fdividef(T - q0, slope);
            int nc = step > 0 ? (int)ceilf(fminf(fmaxf(est, -1.0e6f), 1.0e6f))
                               : (int)floorf(fminf(fmaxf(est, -1.0e6f), 1.0e6f)) + 1;
            nc = min(max(nc, -N + 1), N);
            for (int tries = 0;; ++tries) {
                // q at samples nc - 1 and nc (the band_floor expression) against the
                // integer T: q - T is exact wherever it is below 1 in magnitude, and a side
                // of T is certified when q is at least e from it
                const float da = fmaf(fmaf((float)(nc - 1), a.hf, dv), D[r], fr.tf[r]) - T;
                const float db = fmaf(fmaf((float)nc, a.hf, dv), D[r], fr.tf[r]) - T;
                const bool ok2 = (da >= e[r] || da < -e[r]) && (db >= e[r] || db < -e[r]);
                if (!ok2 || tries > 2) return false;
                const bool at_b = step > 0 ? db >= 0.0f : db < 0.0f;
                const bool at_a = step > 0 ? da >= 0.0f : da < 0.0f;
                if (at_b && !at_a) break;
                if (!at_b) {
                    if (nc >= N) return false;
                    ++nc;
                } else {
                    if (nc <= -N + 1) return false;
                    --nc;
                }
            }
            if (j == 1) n1[r] = nc;
            else n2[r] = nc;
        }
    }
    // the keys in sample order: changes at the same sample make one key
    int k0 = klo[0], k1 = klo[1], k2 = klo[2];
    int c0 = 0, c1 = 0, c2 = 0;  // changes taken per axis
    for (int it = 0;; ++it) {
        const int b0 = fr.Ti[0] + k0, b1 = fr.Ti[1] + k1, b2 = fr.Ti[2] + k2;
        if (key_in_range(a.seg, b0, b1, b2)) push_key(m, rk, pack_key(a.seg, b0, b1, b2), frame);
        else *range_err = true;
        const int x0 = c0 == 0 ? n1[0] : (c0 == 1 ? n2[0] : kNone);
        const int x1 = c1 == 0 ? n1[1] : (c1 == 1 ? n2[1] : kNone);
        const int x2 = c2 == 0 ? n1[2] : (c2 == 1 ? n2[2] : kNone);
        const int n = min(x0, min(x1, x2));
        if (n == kNone || it >= 6) break;
        if (x0 == n) k0 += st[0], ++c0;
        if (x1 == n) k1 += st[1], ++c1;
        if (x2 == n) k2 += st[2], ++c2;
    }
    return true;
}

// Keys of every valid pixel's band samples (reading R1), inserted into the hash.
//
// The key of a sample is floor(t/bs + z D) per axis, D = R (u/fx, v/fy, 1) / bs the
// pixel's ray step per metre of depth in block units and z = d + n h.  It is
// evaluated in float32 with an error bound and certified when no integer lies within
// the bound; otherwise the float64 path in the oracle's operation order decides.
// Per ray: D (rounding error below 2^-21 DA, DA the magnitude of its terms), the
// bound on |z| error ez = 2^-20 (d + N h), and per axis one bound e for all samples,
//   |q - q_real| <= 2^-21 DA (1.25 z + 0.125 N h) + 2^-24 (|q| + 1)
// (rounding of D, of z, of the fma and of t/bs), covered at least twice by
//   e = 2.5 2^-21 DA (z_max + N h) + 2^-22 (q_max + 1),
// q linear in z so that q_max = max |q| over the band's two ends.
//
// The grid strides over 256-pixel tiles of all the call's maps, a tile within one map,
// so that each CTA step reads one pose.  Each map's largest valid depth goes to its
// counter when a CTA leaves the map.
__global__ void __launch_bounds__(256) alloc_keys_kernel(const float* __restrict__ depth, AllocArgs a, DeviceMap m) {
    const int npix = a.W * a.H;
    const int lane = threadIdx.x & 31;
    const float eps = 9.53674316e-7f;  // 2^-20
    const float kMagic = 12582912.0f;  // 1.5 2^23: v + kMagic holds the integer nearest v for |v| < 2^22
    bool range_err = false;
    float dmax = 0.0f;  // largest valid depth seen by this thread in map `dframe`
    int dframe = -1;
    const int n_tiles = a.n_frames * a.tiles;
    // The loop bound is CTA-uniform so every lane reaches the warp collectives.
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int frame = tile / a.tiles;
        if (frame != dframe) {
            for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
            if (lane == 0 && dmax > 0.0f) atomicMax(m.counters + kFrameDepthMax + dframe, __float_as_int(dmax));
            dmax = 0.0f;
            dframe = frame;
        }
        const AllocFrame& fr = a.fr[frame];
        const int pix = (tile - frame * a.tiles) * 256 + (int)threadIdx.x;
        float dv = pix < npix ? __ldg(depth + (size_t)frame * npix + pix) : 0.0f;
        const bool valid = pix < npix && isfinite(dv) && dv > 0.0f;
        if (valid) dmax = fmaxf(dmax, dv);
        const int y = (int)__umul64hi((unsigned long long)(unsigned)pix, a.w_magic), x = pix - y * a.W;
        float D[3] = {0.0f, 0.0f, 0.0f}, e[3] = {0.0f, 0.0f, 0.0f};
        float ez = 0.0f;
        bool fast = false;
        if (valid) {
            // u = (x + 0.5) - cx with cx as hi + lo: relative error below 2^-23
            const float ua = (((float)x + 0.5f) - a.cx_hi) - a.cx_lo;
            const float va = (((float)y + 0.5f) - a.cy_hi) - a.cy_lo;
            const float ax = ua * a.ifx, ay = va * a.ify;
            const float zmax = dv + a.nhf, zmin = dv - a.nhf;
            ez = eps * zmax + 1e-30f;
            fast = true;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                D[r] = fmaf(fr.Rf[3 * r], ax, fmaf(fr.Rf[3 * r + 1], ay, fr.Rf[3 * r + 2])) * a.ibs;
                const float DA = (fabsf(fr.Rf[3 * r] * ax) + fabsf(fr.Rf[3 * r + 1] * ay) + fabsf(fr.Rf[3 * r + 2])) * a.ibs;
                const float qm = fmaxf(fabsf(fmaf(zmin, D[r], fr.tf[r])), fabsf(fmaf(zmax, D[r], fr.tf[r])));
                fast = fast && qm < 2097152.0f;  // beyond 2^21 the float64 path reports the range
                e[r] = fmaf(1.25f * eps, DA * (zmax + a.nhf), 0.25f * eps * (qm + 1.0f));
            }
        }
        // the distinct block keys of this ray's band samples, in sample order (consecutive
        // samples mostly share a block), inserted a warp round at a time once collected;
        // first from the band's ends and floor changes, else sample by sample
        RayKeys rk;
        const bool done = valid && fast && band_keys_by_events(a, fr, frame, dv, D, e, ez, m, rk, &range_err);
        unsigned long long last = kEmptyKey;
        int l0 = INT_MIN, l1 = 0, l2 = 0;  // last certified floor triple (INT_MIN: none)
        float nf = (float)(-a.N);
        for (int n = -a.N; valid && !done && n <= a.N; ++n, nf += 1.0f) {
            unsigned long long key = kEmptyKey;
            bool decided = false;
            if (fast) {
                const float z = fmaf(nf, a.hf, dv);
                if (z < -ez) continue;  // certainly behind the camera
                if (z > ez) {
                    bool ok = true;
                    int k[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const float q = fmaf(z, D[r], fr.tf[r]);
                        const float tq = __fadd_rn(q, kMagic);  // nearest integer n + kMagic
                        const float nq = tq - kMagic;
                        const bool down = nq > q;               // floor(q) = n - 1
                        const float fr = q - (down ? nq - 1.0f : nq);  // q - floor(q), exact
                        ok = ok && fr >= e[r] && 1.0f - fr > e[r];
                        k[r] = __float_as_int(tq) - 0x4B400000 - (down ? 1 : 0);
                    }
                    if (ok) {
                        if (k[0] == l0 && k[1] == l1 && k[2] == l2) continue;  // same block as before
                        l0 = k[0], l1 = k[1], l2 = k[2];
                        const int b0 = fr.Ti[0] + k[0], b1 = fr.Ti[1] + k[1], b2 = fr.Ti[2] + k[2];
                        if (!key_in_range(a.seg, b0, b1, b2)) {
                            range_err = true;
                            continue;
                        }
                        key = pack_key(a.seg, b0, b1, b2);
                        decided = true;
                    }
                }
            }
            if (!decided) {
                key = sample_key(a, fr, x, y, (double)dv, n, &range_err);
                l0 = INT_MIN;
            }
            if (key == kEmptyKey || key == last) continue;
            last = key;
            push_key(m, rk, key, frame);
        }
        warp_insert(m, rk, lane, frame);
    }
    if (range_err) report(m.counters, kErrRange);
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0 && dmax > 0.0f) atomicMax(m.counters + kFrameDepthMax + dframe, __float_as_int(dmax));
}

struct LaserAllocArgs {
    double R[9], t[3];
    double h, bs;   // sample spacing s/2, block size 8 s
    double mu;
    int Ti[3];      // floor(t / bs)
    float tf[3];    // t / bs - Ti, in [0, 1)
    float hf, ibs;  // h, 1/bs as float32
    int N, seg;
    long long n;    // points
};

// Band-sample keys of a laser point (allocation along the ray): samples at range
// rho = r + n h, n = -N..N, rho > 0, key = floor((dg rho + t) / bs) per axis.  The ray
// (r, dg) is set up in float64 in the oracle's order; each sample is evaluated in
// float32 relative to floor(t / bs), q = tf + rho Dg with Dg = dg / bs, and certified
// with one bound per ray and axis,
//   |q - q_real| <= 2^-24 (5 rho_max |Dg| + |q| + 1)   (rounding of dg, 1/bs, the product,
//                                                         r, h, rho, the fma and tf)
//   e = 2^-20 rho_max |Dg| + 2^-21 (q_max + 1)         (at least 3 times that),
// and rho itself against 0 with 2^-22 rho_max (twice its error); otherwise the float64
// path decides.
__global__ void __launch_bounds__(256) laser_keys_kernel(const float* __restrict__ pts, LaserAllocArgs a, DeviceMap m) {
    const int lane = threadIdx.x & 31;
    const float eps20 = 9.53674316e-7f, eps21 = 4.76837158e-7f, eps22 = 2.38418579e-7f;
    bool range_err = false;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < a.n; base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        double r = 0.0, dg[3] = {0.0, 0.0, 0.0};
        bool valid = i < a.n && laser_ray(a.R, __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2),
                                          &r, dg);
        // the range limit of fusion: M = floor((r + mu) / h) < 2^22
        valid = valid && floor(__ddiv_rn(__dadd_rn(r, a.mu), a.h)) < 4194304.0;
        float Dg[3] = {0.0f, 0.0f, 0.0f}, e[3] = {0.0f, 0.0f, 0.0f};
        float rf = 0.0f, erho = 0.0f;
        bool fast = false;
        if (valid) {
            rf = (float)r;
            const float rmax = rf + (float)a.N * a.hf;
            erho = eps22 * rmax + 1e-30f;
            fast = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Dg[k] = (float)dg[k] * a.ibs;
                const float qm = fmaxf(fabsf(fmaf(fmaxf(rf - (float)a.N * a.hf, 0.0f), Dg[k], a.tf[k])),
                                       fabsf(fmaf(rmax, Dg[k], a.tf[k])));
                fast = fast && qm < 2097152.0f;
                e[k] = fmaf(eps20, rmax * fabsf(Dg[k]), eps21 * (qm + 1.0f));
            }
        }
        RayKeys rk;
        unsigned long long last = kEmptyKey;
        float nf = (float)(-a.N);
        for (int n = -a.N; valid && n <= a.N; ++n, nf += 1.0f) {
            unsigned long long key = kEmptyKey;
            bool decided = false;
            if (fast) {
                const float rho = fmaf(nf, a.hf, rf);
                if (rho < -erho) continue;  // behind the sensor for certain
                if (rho > erho) {
                    bool ok = true;
                    int kk[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float q = fmaf(rho, Dg[k], a.tf[k]);
                        const float tq = __fadd_rn(q, 12582912.0f);
                        const float nq = tq - 12582912.0f;
                        const bool down = nq > q;
                        const float fr = q - (down ? nq - 1.0f : nq);
                        ok = ok && fr >= e[k] && 1.0f - fr > e[k];
                        kk[k] = __float_as_int(tq) - 0x4B400000 - (down ? 1 : 0);
                    }
                    if (ok) {
                        const int b0 = a.Ti[0] + kk[0], b1 = a.Ti[1] + kk[1], b2 = a.Ti[2] + kk[2];
                        if (!key_in_range(a.seg, b0, b1, b2)) {
                            range_err = true;
                            continue;
                        }
                        key = pack_key(a.seg, b0, b1, b2);
                        decided = true;
                    }
                }
            }
            if (!decided) {
                const double rho = __dadd_rn(r, __dmul_rn((double)n, a.h));
                if (!(rho > 0.0)) continue;
                double kb[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) kb[k] = floor(__ddiv_rn(__dadd_rn(__dmul_rn(dg[k], rho), a.t[k]), a.bs));
                if (!(kb[0] >= -kCoordBias && kb[0] < kCoordBias && kb[1] >= -kCoordBias && kb[1] < kCoordBias &&
                      kb[2] >= -kCoordBias && kb[2] < kCoordBias)) {
                    range_err = true;
                    continue;
                }
                key = pack_key(a.seg, (int32_t)kb[0], (int32_t)kb[1], (int32_t)kb[2]);
            }
            if (key == last) continue;
            last = key;
            push_key(m, rk, key, 0);
        }
        warp_insert(m, rk, lane, 0);
    }
    if (range_err) report(m.counters, kErrRange);
}

// Sorts (key, val) pairs in place in chunks of CHUNK (bitonic network in shared
// memory over the next power of two >= the chunk's count).  *count may exceed
// capacity; only the first `capacity` pairs exist.  With `birth` (the allocation's new
// keys, val = hash slot), each key's segment bits are first replaced by its slot's
// birth, so that the keys sort by (birth, key) and are stored that way.
template <int CHUNK>
__global__ void __launch_bounds__(1024) sort_chunks_kernel(unsigned long long* keys, uint32_t* vals,
                                                           const int32_t* count, int capacity,
                                                           const int32_t* __restrict__ birth) {
    __shared__ unsigned long long sk[CHUNK];
    __shared__ uint32_t ss[CHUNK];
    const int n = min(*count, capacity);
    const int base = blockIdx.x * CHUNK;
    if (base >= n) return;
    const int cnt = min(CHUNK, n - base);
    int size = 64;
    while (size < cnt) size <<= 1;
    for (int i = threadIdx.x; i < size; i += blockDim.x) {
        unsigned long long k = kEmptyKey;
        uint32_t v = 0u;
        if (i < cnt) {
            k = keys[base + i], v = vals[base + i];
            if (birth) k = ((unsigned long long)birth[v] << kBirthShift) | (k & kCoordMask);
        }
        sk[i] = k;
        ss[i] = v;
    }
    __syncthreads();
    for (int k = 2; k <= size; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < size; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long a = sk[i], b = sk[ixj];
                    if ((a > b) == up) {
                        sk[i] = b;
                        sk[ixj] = a;
                        const uint32_t t = ss[i];
                        ss[i] = ss[ixj];
                        ss[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        keys[base + i] = sk[i];
        vals[base + i] = ss[i];
    }
}

// Global rank of element i among n distinct keys sorted in chunks: its position in
// its own chunk plus, for every other chunk, the number of keys below it.
__device__ long long global_rank(const unsigned long long* keys, int n, int i, int chunk) {
    const unsigned long long key = keys[i];
    const int nchunks = (n + chunk - 1) / chunk;
    const int c = i / chunk;
    long long rank = i - c * chunk;
    for (int c2 = 0; c2 < nchunks; ++c2) {
        if (c2 == c) continue;
        int lo = c2 * chunk, hi = min(lo + chunk, n);
        const int first = lo;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (keys[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        rank += lo - first;
    }
    return rank;
}

__global__ void order_scatter_kernel(const unsigned long long* keys, const uint32_t* vals, const int32_t* count,
                                     int capacity, int32_t* order) {
    const int n = min(*count, capacity);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        order[global_rank(keys, n, i, kSortChunk)] = (int32_t)vals[i];
}

__global__ void rank_assign_kernel(DeviceMap m) {
    const int n = min(m.counters[kNumNew], (int)m.max_new);
    const int nb = m.counters[kNumBlocks];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // the list holds (birth, key without segment); the table holds the key itself
        const unsigned long long sorted = m.new_keys[i];
        const long long idx = nb + global_rank(m.new_keys, n, i, kNewKeyChunk);
        const uint32_t slot = m.new_slots[i];
        if (idx < (long long)m.max_blocks) {
            int32_t s, x, y, z;
            unpack_key(m.hash_keys[slot], &s, &x, &y, &z);
            reinterpret_cast<int4*>(m.coords)[idx] = make_int4(s, x, y, z);
            m.block_birth[idx] = (uint8_t)(sorted >> kBirthShift);
            m.hash_vals[slot] = (int32_t)idx;
        } else {
            m.hash_vals[slot] = -2;
            report(m.counters, kErrPoolFull);
        }
    }
}

__global__ void order_keys_kernel(const int32_t* coords, const int32_t* count, unsigned long long* keys,
                                  uint32_t* vals) {
    const int n = *count;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const int4 k = reinterpret_cast<const int4*>(coords)[b];
        keys[b] = pack_key(k.x, k.y, k.z, k.w);
        vals[b] = (uint32_t)b;
    }
}

struct ZeroRegions {
    char* base[11];
    size_t esize[11];
};

// Zeroes blocks [first, first + count) of every per-voxel field; first/count come from
// the device counters when `from_counters` is set (allocation) or from the arguments.
__global__ void zero_blocks_kernel(DeviceMap m, ZeroRegions z, int nreg, int from_counters, long long first_arg,
                                   long long count_arg) {
    long long first = first_arg, count = count_arg;
    if (from_counters) {
        const int n = min(m.counters[kNumNew], (int)m.max_new);
        first = m.counters[kNumBlocks];
        count = min((long long)n, (long long)m.max_blocks - first);
    }
    if (count <= 0) return;
    for (int r = 0; r < nreg; ++r) {
        const size_t bytes_per_block = (size_t)kBlockVoxels * z.esize[r];
        uint4* p = reinterpret_cast<uint4*>(z.base[r] + (size_t)first * bytes_per_block);
        const size_t n16 = (size_t)count * bytes_per_block / 16;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
            p[i] = make_uint4(0, 0, 0, 0);
    }
}

__global__ void commit_kernel(DeviceMap m) {
    const int inserted = m.counters[kNumNew];
    const int n = min(inserted, (int)m.max_new);
    const int nb = m.counters[kNumBlocks];
    const int added = (int)min((long long)n, (long long)m.max_blocks - nb);
    m.counters[kLastNew] = added;
    m.counters[kNumBlocks] = nb + added;
    m.counters[kNumNew] = 0;
}

__global__ void load_blocks_kernel(DeviceMap m, const int32_t* __restrict__ coords, long long n, long long base) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int4 c = reinterpret_cast<const int4*>(coords)[i];
        if (!key_in_range(c.x, c.y, c.z, c.w)) {
            report(m.counters, kErrRange);
            continue;
        }
        const unsigned long long key = pack_key(c.x, c.y, c.z, c.w);
        const uint32_t h = hash_key(key);
        bool done = false;
        for (int p = 0; p < kMaxProbe && !done; ++p) {
            const uint32_t slot = (h + (uint32_t)p) & m.slot_mask;
            const unsigned long long prev = atomicCAS(m.hash_keys + slot, kEmptyKey, key);
            if (prev == kEmptyKey) {
                m.hash_vals[slot] = (int32_t)(base + i);
                reinterpret_cast<int4*>(m.coords)[base + i] = c;
                done = true;
            } else if (prev == key) {
                report(m.counters, kErrDuplicate);
                done = true;
            }
        }
        if (!done) report(m.counters, kErrHashFull);
    }
}

__global__ void set_count_kernel(DeviceMap m, int32_t n) { m.counters[kNumBlocks] = n; }

ZeroRegions all_regions(denser_ctx* c, int* nreg) {
    ZeroRegions z;
    const size_t mb = (size_t)c->d.max_blocks * kBlockVoxels;
    int r = 0;
    z.base[r] = (char*)c->d.f, z.esize[r++] = 4;
    z.base[r] = (char*)c->d.w, z.esize[r++] = 4;
    z.base[r] = (char*)c->d.u, z.esize[r++] = c->elem_size;
    for (int k = 0; k < 2; ++k) z.base[r] = (char*)c->d.ub[k], z.esize[r++] = c->elem_size;
    for (int k = 0; k < 2; ++k)
        for (int a = 0; a < 3; ++a) z.base[r] = (char*)c->d.p[k] + a * mb * c->elem_size, z.esize[r++] = c->elem_size;
    *nreg = r;
    return z;
}

}  // namespace

int finish_alloc(denser_ctx* c, cudaStream_t s);

int launch_alloc(denser_ctx* c, const float* depth, int n_frames, const denser_intrinsics* K, const double* T,
                 int32_t segment, cudaStream_t s) {
    AllocArgs a;
    a.fx = K->fx, a.fy = K->fy, a.cx = K->cx, a.cy = K->cy;
    a.h = 0.5 * c->prm.voxel_size;
    a.bs = 8.0 * c->prm.voxel_size;
    a.W = K->width, a.H = K->height;
    a.N = (int)ceil(c->prm.mu / a.h - 1e-9);
    a.ifx = (float)(1.0 / a.fx), a.ify = (float)(1.0 / a.fy), a.ibs = (float)(1.0 / a.bs);
    a.cx_hi = (float)a.cx, a.cx_lo = (float)(a.cx - (double)a.cx_hi);
    a.cy_hi = (float)a.cy, a.cy_lo = (float)(a.cy - (double)a.cy_hi);
    a.n_frames = n_frames;
    for (int i = 0; i < n_frames; ++i) {
        AllocFrame& fr = a.fr[i];
        const double* Ti = T + 16 * i;
        for (int r = 0; r < 3; ++r) {
            for (int q = 0; q < 3; ++q) fr.R[3 * r + q] = Ti[4 * r + q];
            fr.t[r] = Ti[4 * r + 3];
        }
        for (int e = 0; e < 9; ++e) fr.Rf[e] = (float)fr.R[e];
        for (int r = 0; r < 3; ++r) {
            const double tb = fr.t[r] / a.bs;
            const double ti = floor(tb);
            fr.Ti[r] = (int)std::max(-2.0 * kCoordBias, std::min(2.0 * kCoordBias, ti));
            fr.tf[r] = (float)(tb - (double)fr.Ti[r]);
        }
    }
    a.hf = (float)a.h;
    a.nhf = (float)(a.N * a.h);
    // floor(n / W) = floor(n * ceil(2^64 / W) / 2^64) for every 32-bit n (W < 2^32)
    a.w_magic = ~0ull / (unsigned long long)a.W + 1ull;
    a.seg = segment;
    const int npix = a.W * a.H;
    a.tiles = (npix + 255) / 256;
    // the fusion of the same maps reads the visible count and the largest valid depths
    // that this pass records (zeroed first, with the words between them)
    cudaMemsetAsync(c->d.counters + kNumVisible, 0, (kCounterWords - kNumVisible) * sizeof(int32_t), s);
    if (c->profile) cudaEventRecord(c->prof_ev[0], s);
    alloc_keys_kernel<<<grid_for(c->sm_count, (int64_t)n_frames * a.tiles * 256, 256, 8), 256, 0, s>>>(depth, a,
                                                                                                        c->d);
    c->launches += 1;
    if (c->profile) cudaEventRecord(c->prof_ev[1], s);
    const int rc = finish_alloc(c, s);
    if (c->profile) cudaEventRecord(c->prof_ev[2], s);
    return rc;
}

// The inserted keys of one allocation call become blocks: sorted (chunks, then ranks
// across chunks), zeroed, counted.
int finish_alloc(denser_ctx* c, cudaStream_t s) {
    const int chunks = (int)((c->d.max_new + kNewKeyChunk - 1) / kNewKeyChunk);
    sort_chunks_kernel<kNewKeyChunk><<<chunks, kNewKeyChunk, 0, s>>>(c->d.new_keys, c->d.new_slots, c->d.counters + kNumNew,
                                               (int)c->d.max_new, c->d.hash_birth);
    rank_assign_kernel<<<grid_for(c->sm_count, c->d.max_new, 256, 4), 256, 0, s>>>(c->d);
    int nreg;
    ZeroRegions z = all_regions(c, &nreg);
    zero_blocks_kernel<<<c->sm_count * 4, 256, 0, s>>>(c->d, z, nreg, 1, 0, 0);
    commit_kernel<<<1, 1, 0, s>>>(c->d);
    c->launches += 4;
    c->nbr_valid_blocks = -1;
    c->order_valid_blocks = -1;
    return cuda_check(c, cudaGetLastError(), "allocation kernels");
}

int launch_alloc_points(denser_ctx* c, const float* pts, int64_t n, const double* T, int32_t segment,
                        cudaStream_t s) {
    LaserAllocArgs a;
    a.h = 0.5 * c->prm.voxel_size;
    a.bs = 8.0 * c->prm.voxel_size;
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) a.R[3 * r + q] = T[4 * r + q];
        a.t[r] = T[4 * r + 3];
        const double tb = a.t[r] / a.bs;
        const double ti = floor(tb);
        a.Ti[r] = (int)std::max(-2.0 * kCoordBias, std::min(2.0 * kCoordBias, ti));
        a.tf[r] = (float)(tb - (double)a.Ti[r]);
    }
    a.N = (int)ceil(c->prm.mu / a.h - 1e-9);
    a.mu = c->prm.mu;
    a.hf = (float)a.h;
    a.ibs = (float)(1.0 / a.bs);
    a.seg = segment;
    a.n = n;
    if (n > 0) {
        laser_keys_kernel<<<grid_for(c->sm_count, n, 256, 8), 256, 0, s>>>(pts, a, c->d);
        c->launches += 1;
    }
    return finish_alloc(c, s);
}

int launch_load_blocks(denser_ctx* c, const int32_t* coords_dev, int64_t n, int64_t base, cudaStream_t s) {
    load_blocks_kernel<<<grid_for(c->sm_count, n, 256, 4), 256, 0, s>>>(c->d, coords_dev, n, base);
    int nreg;
    ZeroRegions z = all_regions(c, &nreg);
    zero_blocks_kernel<<<c->sm_count * 4, 256, 0, s>>>(c->d, z, nreg, 0, base, n);
    set_count_kernel<<<1, 1, 0, s>>>(c->d, (int32_t)(base + n));
    c->launches += 3;
    c->nbr_valid_blocks = -1;
    c->order_valid_blocks = -1;
    return cuda_check(c, cudaGetLastError(), "load_blocks kernels");
}

// Visiting order of the sweep: block indices sorted by key (segment, bz, by, bx).
int launch_block_order(denser_ctx* c, int64_t n_blocks, cudaStream_t s) {
    if (n_blocks <= 0) return DENSER_OK;
    const int32_t* cnt = c->d.counters + kNumBlocks;
    order_keys_kernel<<<grid_for(c->sm_count, n_blocks, 256, 8), 256, 0, s>>>(c->d.coords, cnt, c->order_keys,
                                                                              c->order_vals);
    const int chunks = (int)((n_blocks + kSortChunk - 1) / kSortChunk);
    sort_chunks_kernel<kSortChunk><<<chunks, 1024, 0, s>>>(c->order_keys, c->order_vals, cnt, (int)c->d.max_blocks, nullptr);
    order_scatter_kernel<<<grid_for(c->sm_count, n_blocks, 256, 8), 256, 0, s>>>(c->order_keys, c->order_vals, cnt,
                                                                                 (int)c->d.max_blocks, c->order);
    c->launches += 3;
    c->order_valid_blocks = n_blocks;
    return cuda_check(c, cudaGetLastError(), "block order kernels");
}

int launch_zero_state(denser_ctx* c, int64_t first_block, int64_t n_blocks, cudaStream_t s) {
    int nreg;
    ZeroRegions z = all_regions(c, &nreg);
    // skip f and w (regions 0, 1)
    ZeroRegions zs;
    for (int r = 2; r < nreg; ++r) zs.base[r - 2] = z.base[r], zs.esize[r - 2] = z.esize[r];
    zero_blocks_kernel<<<c->sm_count * 4, 256, 0, s>>>(c->d, zs, nreg - 2, 0, first_block, n_blocks);
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "zero state kernel");
}

}  // namespace denser
