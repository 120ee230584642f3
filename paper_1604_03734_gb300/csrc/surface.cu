// Surface extraction: the zero level set of the regularised u over Omega, as a
// triangle list.  The paper's pipeline hands the regularised model's surface to other
// components (Section II, Fig. 1) without naming an extraction method; this one:
//
//   * a cube is the 2x2x2 voxel centres v + {0,1}^3, meshed only when all eight
//     corners are observed (w > 0, Section III-B): no surface is made up at the border
//     of Omega, where u carries no information;
//   * each cube is split into the six Kuhn tetrahedra around its main diagonal (for a
//     permutation pi of the axes: 0, e_pi0, e_pi0 + e_pi1, (1,1,1)); the split is the
//     same in every cube, so faces shared by neighbouring cubes are cut alike and the
//     mesh has no cracks;
//   * a corner is negative when u < 0 (behind the observed surface); a tetrahedron
//     with one corner alone on its side gives one triangle, two against two give two;
//   * a vertex sits at the linear zero t = u_a / (u_a - u_b) of its edge, measured from
//     the edge's componentwise-lower end a; triangles are wound so that
//     (v1 - v0) x (v2 - v0) points to the non-negative side.
//
// Triangles are ordered by block index, cube (lower corner's local index), tetrahedron
// (lexicographic pi) and triangle within the tetrahedron, so the output is
// deterministic.  Two passes over the blocks: count (per block), exclusive scan, emit.
// A vertex also gets an integer id, (flat voxel index of the lower end) * 8 + direction
// bits, which identifies the edge it lies on: equal ids are the same vertex.
#include "common.cuh"

namespace denser {

namespace {

constexpr int kSurfThreads = 128;  // 4 cubes per thread
constexpr int kR = 9;              // corner region: local coordinates 0..8 on each axis
constexpr int kRegion = kR * kR * kR;

// Kuhn tetrahedra in lexicographic order of pi: corner codes of c1 = e_pi0 and
// c2 = e_pi0 + e_pi1 (bit a = +1 along axis a; c0 = 0, c3 = 7) and the orientation
// sign det[c1, c2, c3] = sign(pi).
__constant__ unsigned char kTetC1[6] = {1, 1, 2, 2, 4, 4};
__constant__ unsigned char kTetC2[6] = {3, 5, 3, 6, 5, 6};
__constant__ signed char kTetSign[6] = {1, -1, -1, 1, 1, -1};

__device__ __forceinline__ int ridx(int x, int y, int z) { return x + kR * (y + kR * z); }

// Number of triangles of a tetrahedron with negative-corner mask m (4 bits).
__device__ __forceinline__ int tet_tris(unsigned m) {
    const int k = __popc(m);
    return k == 2 ? 2 : ((k & 1) ? 1 : 0);
}

struct Region {
    float u[kRegion];
    unsigned char om[kRegion];
    int nbk[8];  // block index of each carry (bit a: the region coordinate along a is 8)
};

// Stages u and Omega on the 9^3 corner region of block b: the block itself and its
// +x, +y, +z, +xy, +xz, +yz and +xyz neighbours' first layers.
template <typename T>
__device__ void load_region(const DeviceMap& m, const T* __restrict__ u, int b, Region& r) {
    const int t = threadIdx.x;
    if (t < 8) {
        int nbk = b;
        if (t > 0) {
            const int4 k = reinterpret_cast<const int4*>(m.coords)[b];
            const long long bx = (long long)k.y + (t & 1), by = (long long)k.z + ((t >> 1) & 1),
                            bz = (long long)k.w + ((t >> 2) & 1);
            nbk = key_in_range(k.x, bx, by, bz) ? hash_lookup(m, pack_key(k.x, (int32_t)bx, (int32_t)by, (int32_t)bz))
                                                : -1;
            if (nbk < 0) nbk = -1;  // pending or rejected slots are not blocks
        }
        r.nbk[t] = nbk;
    }
    __syncthreads();
    for (int i = t; i < kRegion; i += kSurfThreads) {
        const int x = i % kR, y = (i / kR) % kR, z = i / (kR * kR);
        const int carry = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
        const int nbk = r.nbk[carry];
        float uv = 0.0f;
        unsigned char o = 0;
        if (nbk >= 0) {
            const size_t v = (size_t)nbk * kBlockVoxels + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
            o = __ldg(m.w + v) > 0.0f;
            uv = Store<T>::ld(u + v);
        }
        r.u[i] = uv;
        r.om[i] = o;
    }
    __syncthreads();
}

// Negative-corner masks of the six tetrahedra of cube (lx, ly, lz), or 0 for all when
// the cube has an unobserved corner.  Returns the cube's triangle count; fills
// cu[8] with the corner values (corner code order).
__device__ __forceinline__ int cube_case(const Region& r, int lx, int ly, int lz, float* cu, unsigned* neg8) {
    bool all = true;
    unsigned neg = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int i = ridx(lx + (c & 1), ly + ((c >> 1) & 1), lz + ((c >> 2) & 1));
        all = all && r.om[i];
        cu[c] = r.u[i];
        neg |= (cu[c] < 0.0f ? 1u : 0u) << c;
    }
    *neg8 = neg;
    if (!all || neg == 0 || neg == 0xffu) return 0;
    int n = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const unsigned m4 = (neg & 1u) | (((neg >> kTetC1[q]) & 1u) << 1) | (((neg >> kTetC2[q]) & 1u) << 2) |
                            (((neg >> 7) & 1u) << 3);
        n += tet_tris(m4);
    }
    return n;
}

template <typename T>
__global__ void __launch_bounds__(kSurfThreads) surface_count_kernel(DeviceMap m, const T* __restrict__ u,
                                                                     int32_t* __restrict__ counts) {
    __shared__ Region r;
    __shared__ int red[kSurfThreads / 32];
    const int nb = m.counters[kNumBlocks];
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        load_region<T>(m, u, b, r);
        int n = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = 4 * threadIdx.x + q;
            float cu[8];
            unsigned neg;
            n += cube_case(r, l & 7, (l >> 3) & 7, l >> 6, cu, &neg);
        }
        for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
        __syncthreads();
        if (threadIdx.x == 0) counts[b] = red[0] + red[1] + red[2] + red[3];
        __syncthreads();  // r and red are rewritten by the next block
    }
}

// offsets[b] = sum of counts[0..b); offsets[nb] = total.  One CTA of 1024 threads:
// each thread sums a contiguous chunk, the CTA scans the chunk sums, each thread
// writes its chunk's running sums.
__global__ void __launch_bounds__(1024) surface_scan_kernel(const DeviceMap m, const int32_t* __restrict__ counts,
                                                            long long* __restrict__ offsets) {
    __shared__ long long part[1024];
    const int nb = m.counters[kNumBlocks];
    const int t = threadIdx.x;
    const int chunk = (nb + 1023) / 1024;
    const int lo = min(nb, t * chunk), hi = min(nb, lo + chunk);
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {  // Hillis-Steele inclusive scan
        const long long v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (int i = lo; i < hi; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    if (t == 1023) offsets[nb] = part[1023];
}

// Vertex on the edge from tetrahedron corner code ca (lower) to cb of cube (lx, ly, lz).
__device__ __forceinline__ void emit_vertex(const Region& r, int4 key, float s, int lx, int ly, int lz, int ca, int cb,
                                            float ua, float ub, float* pos, long long* id) {
    const int ox = lx + (ca & 1), oy = ly + ((ca >> 1) & 1), oz = lz + ((ca >> 2) & 1);
    const int dir = ca ^ cb;
    const float t = ua / (ua - ub);
    pos[0] = ((float)(8 * key.y + ox) + 0.5f + ((dir & 1) ? t : 0.0f)) * s;
    pos[1] = ((float)(8 * key.z + oy) + 0.5f + ((dir & 2) ? t : 0.0f)) * s;
    pos[2] = ((float)(8 * key.w + oz) + 0.5f + ((dir & 4) ? t : 0.0f)) * s;
    const int carry = (ox >> 3) | ((oy >> 3) << 1) | ((oz >> 3) << 2);
    const long long flat = (long long)r.nbk[carry] * kBlockVoxels + (ox & 7) + 8 * (oy & 7) + 64 * (oz & 7);
    *id = flat * 8 + dir;
}

template <typename T>
__global__ void __launch_bounds__(kSurfThreads) surface_emit_kernel(DeviceMap m, const T* __restrict__ u,
                                                                    const long long* __restrict__ offsets, float s,
                                                                    long long capacity, float* __restrict__ tri_pos,
                                                                    long long* __restrict__ tri_ids) {
    __shared__ Region r;
    __shared__ int wsum[kSurfThreads / 32];
    const int nb = m.counters[kNumBlocks];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        load_region<T>(m, u, b, r);
        const int4 key = reinterpret_cast<const int4*>(m.coords)[b];
        int cnt[4];
        int n = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = 4 * threadIdx.x + q;
            float cu[8];
            unsigned neg;
            cnt[q] = cube_case(r, l & 7, (l >> 3) & 7, l >> 6, cu, &neg);
            n += cnt[q];
        }
        // exclusive scan of the per-thread counts in thread (= cube) order
        int inc = n;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int base = 0;
        for (int w = 0; w < warp; ++w) base += wsum[w];
        long long out = offsets[b] + base + inc - n;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            if (cnt[q] == 0) continue;
            const int l = 4 * threadIdx.x + q;
            const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
            float cu[8];
            unsigned neg;
            cube_case(r, lx, ly, lz, cu, &neg);
#pragma unroll 1
            for (int q6 = 0; q6 < 6; ++q6) {
                const int code[4] = {0, kTetC1[q6], kTetC2[q6], 7};
                unsigned m4 = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) m4 |= ((neg >> code[i]) & 1u) << i;
                const int k = __popc(m4);
                if (k == 0 || k == 4) continue;
                // edges (i, j), i < j, of the (up to) two triangles, wound per the header
                int e[2][3][2];
                int ntri;
                if (k & 1) {
                    const int lone = __ffs(k == 1 ? m4 : (~m4 & 15u)) - 1;
                    // the other three in the order of an even permutation that puts the
                    // lone corner first: the triangle's normal then points away from it on a
                    // positively oriented tetrahedron
                    const int o0 = lone == 0 ? 1 : (lone == 1 ? 0 : (lone == 2 ? 3 : 2));
                    const int o1 = lone == 0 ? 2 : (lone == 1 ? 3 : (lone == 2 ? 0 : 1));
                    const int o2 = lone == 0 ? 3 : (lone == 1 ? 2 : (lone == 2 ? 1 : 0));
                    const bool flip = (kTetSign[q6] > 0) != (k == 1);
                    const int oo[3] = {o0, flip ? o2 : o1, flip ? o1 : o2};
#pragma unroll
                    for (int v = 0; v < 3; ++v) {
                        e[0][v][0] = min(lone, oo[v]);
                        e[0][v][1] = max(lone, oo[v]);
                    }
                    ntri = 1;
                } else {
                    const int A = __ffs(m4) - 1, B = 31 - __clz(m4);
                    const unsigned pm = ~m4 & 15u;
                    const int C = __ffs(pm) - 1, D = 31 - __clz(pm);
                    // parity of (A, B, C, D) as a permutation of (0, 1, 2, 3): odd exactly
                    // for the negative pairs {0, 2} and {1, 3}
                    const int par = (m4 == 5u || m4 == 10u) ? -1 : 1;
                    const bool flip = kTetSign[q6] * par < 0;
                    const int t0[3][2] = {{A, C}, {A, D}, {B, D}};
                    const int t1[3][2] = {{A, C}, {B, D}, {B, C}};
#pragma unroll
                    for (int v = 0; v < 3; ++v) {
                        const int vv = flip ? (v == 0 ? 0 : 3 - v) : v;
                        e[0][v][0] = min(t0[vv][0], t0[vv][1]);
                        e[0][v][1] = max(t0[vv][0], t0[vv][1]);
                        e[1][v][0] = min(t1[vv][0], t1[vv][1]);
                        e[1][v][1] = max(t1[vv][0], t1[vv][1]);
                    }
                    ntri = 2;
                }
                for (int tr = 0; tr < ntri; ++tr, ++out) {
                    if (out >= capacity) continue;
                    float pos[9];
                    long long id[3];
#pragma unroll
                    for (int v = 0; v < 3; ++v) {
                        const int i = e[tr][v][0], j = e[tr][v][1];
                        emit_vertex(r, key, s, lx, ly, lz, code[i], code[j], cu[code[i]], cu[code[j]], pos + 3 * v,
                                    id + v);
                    }
                    if (tri_pos) {
                        float* dst = tri_pos + out * 9;
#pragma unroll
                        for (int v = 0; v < 9; ++v) dst[v] = pos[v];
                    }
                    if (tri_ids) {
                        long long* dst = tri_ids + out * 3;
                        dst[0] = id[0], dst[1] = id[1], dst[2] = id[2];
                    }
                }
            }
        }
        __syncthreads();  // r and wsum are rewritten by the next block
    }
}

template <typename T>
int surface_launch(denser_ctx* c, int64_t nb, int pass, float* tri_pos, long long* tri_ids, int64_t capacity,
                   cudaStream_t s) {
    const int grid = (int)std::min<int64_t>(nb, (int64_t)c->sm_count * 8);
    if (pass == 0) {
        surface_count_kernel<T><<<grid, kSurfThreads, 0, s>>>(c->d, (const T*)c->d.u, c->surf_counts);
        surface_scan_kernel<<<1, 1024, 0, s>>>(c->d, c->surf_counts, c->surf_offsets);
        c->launches += 2;
    } else {
        surface_emit_kernel<T><<<grid, kSurfThreads, 0, s>>>(c->d, (const T*)c->d.u, c->surf_offsets,
                                                             (float)c->prm.voxel_size, capacity, tri_pos, tri_ids);
        c->launches += 1;
    }
    return cuda_check(c, cudaGetLastError(), "surface kernel");
}

}  // namespace

// pass 0: count per block and scan into c->surf_offsets (offsets[nb] = total);
// pass 1: write the first `capacity` triangles.
int launch_surface(denser_ctx* c, int64_t nb, int pass, float* tri_pos, long long* tri_ids, int64_t capacity,
                   cudaStream_t s) {
    if (nb <= 0) return DENSER_OK;
    switch (c->prm.precision) {
        case DENSER_FP16: return surface_launch<__half>(c, nb, pass, tri_pos, tri_ids, capacity, s);
        case DENSER_BF16: return surface_launch<__nv_bfloat16>(c, nb, pass, tri_pos, tri_ids, capacity, s);
        default: return surface_launch<float>(c, nb, pass, tri_pos, tri_ids, capacity, s);
    }
}

}  // namespace denser
