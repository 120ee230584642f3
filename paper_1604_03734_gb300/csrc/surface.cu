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
// deterministic.  Passes: upper-neighbour lookup; count (per block), which also lists
// every cube with triangles; exclusive scan of the counts; emit, one thread per listed
// cube.
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

// Block index of each upper neighbour (carry code c: +x for bit 0, +y bit 1, +z bit 2;
// entry 0 is the block itself), -1 where unallocated: 8 int32 per block.  One thread
// per lookup, so that the hash probes of all blocks overlap.
__global__ void surface_nbr_kernel(DeviceMap m, int32_t* __restrict__ up) {
    const int nb = m.counters[kNumBlocks];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nb * 8;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i >> 3), c = (int)(i & 7);
        int nbk = b;
        if (c) {
            const int4 k = reinterpret_cast<const int4*>(m.coords)[b];
            const long long bx = (long long)k.y + (c & 1), by = (long long)k.z + ((c >> 1) & 1),
                            bz = (long long)k.w + ((c >> 2) & 1);
            nbk = key_in_range(k.x, bx, by, bz) ? hash_lookup(m, pack_key(k.x, (int32_t)bx, (int32_t)by, (int32_t)bz))
                                                : -1;
            if (nbk < 0) nbk = -1;  // pending or rejected slots are not blocks
        }
        up[i] = nbk;
    }
}

// Negative-corner mask (bit i: tetrahedron corner i) of Kuhn tetrahedron q of a cube
// whose corner c is negative when bit c of neg8 is set.
__device__ __forceinline__ unsigned tet_mask(unsigned neg8, int q) {
    return (neg8 & 1u) | (((neg8 >> kTetC1[q]) & 1u) << 1) | (((neg8 >> kTetC2[q]) & 1u) << 2) |
           (((neg8 >> 7) & 1u) << 3);
}

// Count pass.  Each thread takes four consecutive cubes along x (their 20 corners are
// read once), finds each cube's negative-corner mask and whether all eight corners are
// observed, and takes the cube's triangle count from a 256-entry table.  Per block:
// counts[b] = the block's triangles; every cube with triangles is appended to `list`
// as (block << 32 | cube << 23 | mask << 15 | first triangle within the block), in
// cube order within the block (the blocks' chunks land in any order).  *cursor counts
// the entries; entries beyond `cap` are not written (the host then grows the list and
// runs the pass again).
template <typename T>
__global__ void __launch_bounds__(kSurfThreads, 12) surface_count_kernel(DeviceMap m, const T* __restrict__ u,
                                                                         const int32_t* __restrict__ up,
                                                                         int32_t* __restrict__ counts,
                                                                         unsigned long long* __restrict__ list,
                                                                         long long cap,
                                                                         unsigned long long* __restrict__ cursor) {
    __shared__ float su[kRegion];
    __shared__ unsigned char som[kRegion];
    __shared__ int nbk[2][8];  // this block's and the next block's upper neighbours
    __shared__ unsigned char lut[256];  // triangles of a cube by its negative-corner mask
    __shared__ int wsum[kSurfThreads / 32];
    __shared__ unsigned long long chunk;
    const int nb = m.counters[kNumBlocks];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int i = t; i < 256; i += kSurfThreads) {
        int n = 0;
        if (i != 0 && i != 255)
            for (int q = 0; q < 6; ++q) n += tet_tris(tet_mask((unsigned)i, q));
        lut[i] = (unsigned char)n;
    }
    const int lx0 = (4 * t) & 7, ly = ((4 * t) >> 3) & 7, lz = (4 * t) >> 6;
    // the next block's neighbour row is read one block ahead, so that a block's region
    // loads do not wait behind it
    int cur = 0;
    if (t < 8 && (int)blockIdx.x < nb) nbk[0][t] = __ldg(up + 8 * (size_t)blockIdx.x + t);
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int bn = b + gridDim.x;
        const int pre = (t < 8 && bn < nb) ? __ldg(up + 8 * (size_t)bn + t) : -1;
        __syncthreads();
        // the corner region: the block's own rows in halves of four voxels (one per thread,
        // w as one 16-byte load), then 115 items for the upper faces and edges: the +x plane
        // voxel by voxel, the +y and +z planes and the (+y,+z) edge in halves of rows, the
        // (+x,+y) and (+x,+z) edges voxel by voxel, and the far corner
        {
            const int r = t >> 1, hx = 4 * (t & 1), y = r & 7, z = r >> 3;
            const size_t v = (size_t)nbk[cur][0] * kBlockVoxels + hx + 8 * y + 64 * z;
            const float4 w4 = __ldg(reinterpret_cast<const float4*>(m.w + v));
            const int d = ridx(hx, y, z);
            su[d] = Store<T>::ld(u + v), su[d + 1] = Store<T>::ld(u + v + 1);
            su[d + 2] = Store<T>::ld(u + v + 2), su[d + 3] = Store<T>::ld(u + v + 3);
            som[d] = w4.x > 0.0f, som[d + 1] = w4.y > 0.0f, som[d + 2] = w4.z > 0.0f, som[d + 3] = w4.w > 0.0f;
        }
        if (t < 115) {
            // item -> first region voxel (x, y, z), source block (upper-neighbour code), count
            int x, y, z, sel, n;
            if (t < 64) x = 8, y = t & 7, z = t >> 3, sel = 1, n = 1;
            else if (t < 80) x = 4 * (t & 1), y = 8, z = (t - 64) >> 1, sel = 2, n = 4;
            else if (t < 96) x = 4 * (t & 1), y = (t - 80) >> 1, z = 8, sel = 4, n = 4;
            else if (t < 104) x = 8, y = 8, z = t - 96, sel = 3, n = 1;
            else if (t < 112) x = 8, y = t - 104, z = 8, sel = 5, n = 1;
            else if (t < 114) x = 4 * (t & 1), y = 8, z = 8, sel = 6, n = 4;
            else x = 8, y = 8, z = 8, sel = 7, n = 1;
            const int nk = nbk[cur][sel];
            const int d = ridx(x, y, z);
            const size_t v = (size_t)(nk >= 0 ? nk : 0) * kBlockVoxels + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
            for (int k = 0; k < n; ++k) {
                float uv = 0.0f;
                unsigned char o = 0;
                if (nk >= 0) {
                    o = __ldg(m.w + v + k) > 0.0f;
                    uv = Store<T>::ld(u + v + k);
                }
                su[d + k] = uv;
                som[d + k] = o;
            }
        }
        __syncthreads();
        // rows (y, z), (y+1, z), (y, z+1), (y+1, z+1) of x = lx0 .. lx0 + 4: 5-bit masks
        unsigned negr[4], omr[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int base = ridx(lx0, ly + (r & 1), lz + (r >> 1));
            unsigned nm = 0, om = 0;
#pragma unroll
            for (int x = 0; x < 5; ++x) {
                nm |= (su[base + x] < 0.0f ? 1u : 0u) << x;
                om |= (som[base + x] ? 1u : 0u) << x;
            }
            negr[r] = nm;
            omr[r] = om;
        }
        unsigned neg8[4];
        int cnt[4], n = 0, items = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // corner c = (x bit, y bit, z bit): row r = c >> 1, x offset c & 1
            unsigned ng = 0, ob = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                ng |= ((negr[r] >> q) & 3u) << (2 * r);
                ob |= ((omr[r] >> q) & 3u) << (2 * r);
            }
            neg8[q] = ng;
            cnt[q] = ob == 0xffu ? lut[ng] : 0;
            n += cnt[q];
            items += cnt[q] ? 1 : 0;
        }
        // exclusive scan of (cubes listed, triangles) in thread (= cube) order, packed
        const int packed = (items << 16) | n;
        int inc = packed;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < kSurfThreads / 32; ++w) {
            before += w < warp ? wsum[w] : 0;
            total += wsum[w];
        }
        if (t == 0) {
            counts[b] = total & 0xffff;
            chunk = (total >> 16) ? atomicAdd(cursor, (unsigned long long)(total >> 16)) : 0ull;
        }
        __syncthreads();
        const int ex = before + inc - packed;
        long long slot = (long long)chunk + (ex >> 16);
        int tri = ex & 0xffff;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!cnt[q]) continue;
            if (slot < cap)
                list[slot] = ((unsigned long long)(unsigned)b << 32) | ((unsigned long long)(4 * t + q) << 23) |
                             ((unsigned long long)neg8[q] << 15) | (unsigned long long)tri;
            ++slot;
            tri += cnt[q];
        }
        if (t < 8) nbk[cur ^ 1][t] = pre;
        __syncthreads();  // shared state is rewritten by the next block
        cur ^= 1;
    }
}

// offsets[b] = sum of counts[0..b); offsets[nb] = total.  One CTA of 1024 threads walks
// the counts in tiles of 4096: each thread reads four consecutive counts (one 16-byte
// load; counts is 16-byte aligned), the warps scan their 128 counts with shuffles, one
// warp scans the 32 warp totals, and each thread writes its four offsets; the tile's
// total carries into the next tile.
__global__ void __launch_bounds__(1024) surface_scan_kernel(const DeviceMap m, const int32_t* __restrict__ counts,
                                                            long long* __restrict__ offsets) {
    __shared__ long long wsum[32];
    __shared__ long long carry_s;
    const int nb = m.counters[kNumBlocks];
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    long long carry = 0;
    for (int tile = 0; tile < nb; tile += 4096) {
        const int i0 = tile + 4 * t;
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        if (i0 + 3 < nb) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(counts + i0));
            c0 = v.x, c1 = v.y, c2 = v.z, c3 = v.w;
        } else {
            if (i0 < nb) c0 = counts[i0];
            if (i0 + 1 < nb) c1 = counts[i0 + 1];
            if (i0 + 2 < nb) c2 = counts[i0 + 2];
        }
        const long long s4 = (long long)c0 + c1 + c2 + c3;
        long long inc = s4;  // inclusive scan of the four-count sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) wsum[wp] = inc;
        __syncthreads();
        if (wp == 0) {
            long long w = wsum[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            wsum[lane] = wi - w;  // exclusive over the warps
            if (lane == 31) carry_s = wi;
        }
        __syncthreads();
        long long run = carry + wsum[wp] + inc - s4;  // offset of count i0
        if (i0 < nb) offsets[i0] = run;
        run += c0;
        if (i0 + 1 < nb) offsets[i0 + 1] = run;
        run += c1;
        if (i0 + 2 < nb) offsets[i0 + 2] = run;
        run += c2;
        if (i0 + 3 < nb) offsets[i0 + 3] = run;
        carry += carry_s;
        __syncthreads();  // wsum and carry_s are rewritten by the next tile
    }
    if (t == 0) offsets[nb] = carry;
}

// The edges (i, j), i < j, of the triangles of a tetrahedron with negative-corner mask
// m4 and orientation sign sg, wound so that (v1 - v0) x (v2 - v0) points to the
// non-negative side; returns the triangle count.
__device__ __forceinline__ int tet_edges(unsigned m4, int sg, int e[2][3][2]) {
    const int k = __popc(m4);
    if (k & 1) {
        const int lone = __ffs(k == 1 ? m4 : (~m4 & 15u)) - 1;
        // the other three in the order of an even permutation that puts the lone corner
        // first: on a positively oriented tetrahedron the triangle's normal then points
        // away from it
        const int o0 = lone == 0 ? 1 : (lone == 1 ? 0 : (lone == 2 ? 3 : 2));
        const int o1 = lone == 0 ? 2 : (lone == 1 ? 3 : (lone == 2 ? 0 : 1));
        const int o2 = lone == 0 ? 3 : (lone == 1 ? 2 : (lone == 2 ? 1 : 0));
        const bool flip = (sg > 0) != (k == 1);
        const int oo[3] = {o0, flip ? o2 : o1, flip ? o1 : o2};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            e[0][v][0] = min(lone, oo[v]);
            e[0][v][1] = max(lone, oo[v]);
        }
        return 1;
    }
    const int A = __ffs(m4) - 1, B = 31 - __clz(m4);
    const unsigned pm = ~m4 & 15u;
    const int C = __ffs(pm) - 1, D = 31 - __clz(pm);
    // parity of (A, B, C, D) as a permutation of (0, 1, 2, 3): odd exactly for the
    // negative pairs {0, 2} and {1, 3}
    const int par = (m4 == 5u || m4 == 10u) ? -1 : 1;
    const bool flip = sg * par < 0;
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
    return 2;
}

// A listed cube's data, staged per lane of a warp for the emit pass.
struct EmitCube {
    float cu[8];         // u at the eight corners
    long long flat[8];   // flat voxel index of each corner
    float g[3];          // voxel-unit position of corner 0 (+ 1/2)
    unsigned neg8;       // negative-corner mask
    long long out0;      // output index of the cube's first triangle
};

// Emit pass, one warp per 32 listed cubes.  Each lane reads its cube (eight corner
// values, from the block and its upper neighbours) and counts its triangles; then the
// warp's triangles, in output order, are dealt out one per lane: each lane computes one
// triangle of whichever cube holds it (from the staged cube data) into a shared-memory
// slot, and the warp writes the slots back as consecutive words, so that triangles that
// are consecutive in the output (a block's cubes are) go out in whole sectors.  The
// triangles of a cube come from its six tetrahedra in order, from the block's first
// triangle plus the cube's offset.  With n_items_dev, the count is read on the device
// (the count pass queued just before), and nothing is written when the list overflowed
// (more than list_cap cubes: the host then grows the list and runs both passes again).
template <typename T>
__global__ void __launch_bounds__(64) surface_emit_kernel(DeviceMap m, const T* __restrict__ u,
                                                           const int32_t* __restrict__ up,
                                                           const unsigned long long* __restrict__ list,
                                                           long long n_items,
                                                           const unsigned long long* __restrict__ n_items_dev,
                                                           long long list_cap, const long long* __restrict__ offsets,
                                                           float s, long long capacity, float* __restrict__ tri_pos,
                                                           long long* __restrict__ tri_ids) {
    __shared__ EmitCube cubes[2][32];
    __shared__ int first[2][33];          // prefix sums of the lanes' triangle counts
    __shared__ float spos[2][32 * 9];
    __shared__ long long sids[2][32 * 3];
    __shared__ long long sout[2][32];
    if (n_items_dev) {
        n_items = (long long)*n_items_dev;
        if (n_items > list_cap) return;
    }
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    EmitCube* cb = cubes[wp];
    for (long long base = ((long long)blockIdx.x * 2 + wp) * 32; base < n_items; base += (long long)gridDim.x * 64) {
        const long long it = base + lane;
        int ntri = 0;
        if (it < n_items) {
            const unsigned long long w = list[it];
            const int b = (int)(w >> 32);
            const int l = (int)((w >> 23) & 511u);
            const unsigned neg8 = (unsigned)((w >> 15) & 255u);
            const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
            const int4 key = reinterpret_cast<const int4*>(m.coords)[b];
            const int4 u0 = __ldg(reinterpret_cast<const int4*>(up) + 2 * (size_t)b);
            const int4 u1 = __ldg(reinterpret_cast<const int4*>(up) + 2 * (size_t)b + 1);
            EmitCube& c = cb[lane];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int ox = lx + (k & 1), oy = ly + ((k >> 1) & 1), oz = lz + ((k >> 2) & 1);
                // the corner's block: the cube's own or one of its upper neighbours (selects,
                // so that the runtime index keeps the row in registers)
                const int sel = (ox >> 3) | ((oy >> 3) << 1) | ((oz >> 3) << 2);
                const int nk = sel < 4 ? (sel < 2 ? (sel ? u0.y : u0.x) : (sel == 2 ? u0.z : u0.w))
                                       : (sel < 6 ? (sel == 4 ? u1.x : u1.y) : (sel == 6 ? u1.z : u1.w));
                const long long f = (long long)nk * kBlockVoxels + (ox & 7) + 8 * (oy & 7) + 64 * (oz & 7);
                c.flat[k] = f;
                c.cu[k] = Store<T>::ld(u + f);
            }
            c.g[0] = (float)(8 * key.y + lx) + 0.5f;
            c.g[1] = (float)(8 * key.z + ly) + 0.5f;
            c.g[2] = (float)(8 * key.w + lz) + 0.5f;
            c.neg8 = neg8;
            c.out0 = offsets[b] + (long long)(w & 32767u);
#pragma unroll
            for (int q = 0; q < 6; ++q) ntri += tet_tris(tet_mask(neg8, q));
        }
        // exclusive prefix of the lanes' counts
        int inc = ntri;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        first[wp][lane + 1] = inc;
        if (lane == 0) first[wp][0] = 0;
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        __syncwarp();
        for (int j0 = 0; j0 < total; j0 += 32) {
            const int j = j0 + lane;
            const int cnt = min(32, total - j0);
            if (j < total) {
                // the cube holding the warp's triangle j, and which of its triangles
                int lo = 0, hi = 31;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (first[wp][mid] <= j) lo = mid;
                    else hi = mid - 1;
                }
                const EmitCube& c = cb[lo];
                int r = j - first[wp][lo];
                const long long out = c.out0 + r;
                int q = 0, tr = 0;
#pragma unroll 1
                for (; q < 6; ++q) {
                    const int k = tet_tris(tet_mask(c.neg8, q));
                    if (r < k) {
                        tr = r;
                        break;
                    }
                    r -= k;
                }
                const unsigned m4 = tet_mask(c.neg8, q);
                const int c1 = kTetC1[q], c2 = kTetC2[q];
                auto code = [&](int jj) { return jj == 0 ? 0 : (jj == 1 ? c1 : (jj == 2 ? c2 : 7)); };
                int e[2][3][2];
                tet_edges(m4, kTetSign[q], e);
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    // the vertex on the edge from corner ca (the lower end) to cb
                    const int ca = code(tr ? e[1][v][0] : e[0][v][0]), cbn = code(tr ? e[1][v][1] : e[0][v][1]);
                    const int dir = ca ^ cbn;
                    const float ua = c.cu[ca], ub = c.cu[cbn];
                    const float tt = ua / (ua - ub);
                    spos[wp][9 * lane + 3 * v + 0] = (c.g[0] + (float)(ca & 1) + ((dir & 1) ? tt : 0.0f)) * s;
                    spos[wp][9 * lane + 3 * v + 1] = (c.g[1] + (float)((ca >> 1) & 1) + ((dir & 2) ? tt : 0.0f)) * s;
                    spos[wp][9 * lane + 3 * v + 2] = (c.g[2] + (float)((ca >> 2) & 1) + ((dir & 4) ? tt : 0.0f)) * s;
                    sids[wp][3 * lane + v] = c.flat[ca] * 8 + dir;
                }
                sout[wp][lane] = out;
            }
            __syncwarp();
            // consecutive words of the staged triangles to their output places
            if (tri_pos)
                for (int wd = lane; wd < 9 * cnt; wd += 32) {
                    const int t = wd / 9;
                    const long long o = sout[wp][t];
                    if (o < capacity) tri_pos[o * 9 + (wd - 9 * t)] = spos[wp][wd];
                }
            if (tri_ids)
                for (int wd = lane; wd < 3 * cnt; wd += 32) {
                    const int t = wd / 3;
                    const long long o = sout[wp][t];
                    if (o < capacity) tri_ids[o * 3 + (wd - 3 * t)] = sids[wp][wd];
                }
            __syncwarp();
        }
        __syncwarp();  // the staged cubes are rewritten for the next 32
    }
}

template <typename T>
int surface_launch(denser_ctx* c, int64_t nb, int pass, float* tri_pos, long long* tri_ids, int64_t capacity,
                   cudaStream_t s) {
    if (pass == 0) {
        surface_nbr_kernel<<<grid_for(c->sm_count, nb * 8, 256, 8), 256, 0, s>>>(c->d, c->surf_up);
        const int grid = (int)std::min<int64_t>(nb, (int64_t)c->sm_count * 12);
        cudaMemsetAsync(c->surf_cursor, 0, sizeof(unsigned long long), s);
        surface_count_kernel<T><<<grid, kSurfThreads, 0, s>>>(c->d, (const T*)c->d.u, c->surf_up, c->surf_counts,
                                                              c->surf_list, c->surf_list_cap, c->surf_cursor);
        surface_scan_kernel<<<1, 1024, 0, s>>>(c->d, c->surf_counts, c->surf_offsets);
        c->launches += 3;
    } else if (pass == 1) {
        const long long n_items = c->surf_items;
        if (n_items > 0) {
            // small CTAs: a few tens of thousands of listed cubes still spread over every SM
            surface_emit_kernel<T><<<(unsigned)std::max<long long>(1, (n_items + 63) / 64), 64, 0, s>>>(
                c->d, (const T*)c->d.u, c->surf_up, c->surf_list, n_items, nullptr, 0, c->surf_offsets,
                (float)c->prm.voxel_size, capacity, tri_pos, tri_ids);
            c->launches += 1;
        }
    } else {
        // the count still on the device: one warp per 32 entries of the list's capacity
        // (the warps past the count return at once), so that every listed cube starts at once
        const long long grid = std::max<long long>(1, std::min<long long>((c->surf_list_cap + 63) / 64, 1ll << 30));
        surface_emit_kernel<T><<<(unsigned)grid, 64, 0, s>>>(
            c->d, (const T*)c->d.u, c->surf_up, c->surf_list, 0, c->surf_cursor, c->surf_list_cap, c->surf_offsets,
            (float)c->prm.voxel_size, capacity, tri_pos, tri_ids);
        c->launches += 1;
    }
    return cuda_check(c, cudaGetLastError(), "surface kernel");
}

}  // namespace

// pass 0: neighbour rows, counts per block, the list of cubes with triangles, and the
// scan into c->surf_offsets (offsets[nb] = total, *c->surf_cursor = listed cubes);
// pass 1: write the first `capacity` triangles of the c->surf_items listed cubes;
// pass 2: the same with the listed cubes counted on the device (right after pass 0,
// no host round trip between them).
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
