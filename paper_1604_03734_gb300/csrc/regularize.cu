// Omega-aware primal-dual regularisation (Section III-B, Eq. 3 and Eq. 4; Section III-C).
//
// Per regularisation call:
//   omega_bits   Omega = {w > 0} packed 32 voxels per word (ballot per warp);
//   neighbours   per block the indices of its 6 face and 6 (low, high) edge
//                neighbours through the hash table (-1: unallocated = Omega-bar);
// per iteration, one fused sweep.  Each CTA takes one 8^3 block at a time (grid-stride)
// and stages what the block's stencil reads in shared memory: u_bar on the block, its six
// faces and six edges, Omega on the same positions and p on its three low faces (the
// "block as a grid whose boundary conditions come from its neighbours' I_Omega",
// Section III-B).  It takes the dual step on the block and on its low faces (the
// divergence needs p^{k+1} one voxel behind), synchronises, and takes the primal step
// and the relaxation.  u_bar and p are ping-ponged across iterations; u is updated in
// place.  Variants (the schedule picks one; all give bit-identical iterates):
//   sweep_kernel           512 threads, one voxel per thread, stage then compute;
//   sweep_pipe_kernel      the same with cp.async prefetch of the next block;
//   sweep_rows_kernel      64 threads, one 8-voxel x-row per thread in registers; with
//                          ASYNC (the default) the halos are copied by cp.async straight
//                          into shared memory while the block's own rows load;
//   sweep_rows_tma_kernel  the row kernel with the next block's own fields brought in by
//                          1-D bulk copies (TMA) into a double-buffered stage;
//   sweep_rows_kernel<.., BAL>  the row kernel with the face halos split into balanced
//                          items over all threads (asynchronous or through registers).
// and on demand:
//   energy       FP64 primal P(u) and dual D(p) partial sums per CTA (fixed grid, fixed
//                order: deterministic), then one CTA sums the partials.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace denser {

namespace {

constexpr int kTile = 10;  // u_bar / Omega tile: local coordinates -1..8
constexpr int kPTile = 9;  // p tile: local coordinates -1..7
constexpr int kHalo = 432; // 6 faces x 64 + 6 edges x 8
constexpr int kLowHalo = 192;

__device__ inline int t10(int x, int y, int z) { return (x + 1) + kTile * (y + 1) + kTile * kTile * (z + 1); }
__device__ inline int t9(int x, int y, int z) { return (x + 1) + kPTile * (y + 1) + kPTile * kPTile * (z + 1); }
__device__ inline int lin(int x, int y, int z) { return x + 8 * y + 64 * z; }

struct HaloPos {
    int slot;        // neighbour-table entry
    int src;         // voxel offset inside the neighbour block
    int tx, ty, tz;  // tile position
    bool low;        // a low face: p is staged too
};

// Halo entry hid in [0, 432): faces +x, -x, +y, -y, +z, -z (64 each), then the edges
// (-x,+y), (-x,+z), (-y,+x), (-y,+z), (-z,+x), (-z,+y) (8 each).
__device__ inline HaloPos halo_pos(int hid) {
    HaloPos h;
    h.low = false;
    if (hid < 384) {
        const int face = hid >> 6, a = hid & 7, b = (hid >> 3) & 7;
        switch (face) {
            case 0: h.slot = 0, h.src = lin(0, a, b), h.tx = 8, h.ty = a, h.tz = b; break;
            case 1: h.slot = 3, h.src = lin(7, a, b), h.tx = -1, h.ty = a, h.tz = b, h.low = true; break;
            case 2: h.slot = 1, h.src = lin(a, 0, b), h.tx = a, h.ty = 8, h.tz = b; break;
            case 3: h.slot = 4, h.src = lin(a, 7, b), h.tx = a, h.ty = -1, h.tz = b, h.low = true; break;
            case 4: h.slot = 2, h.src = lin(a, b, 0), h.tx = a, h.ty = b, h.tz = 8; break;
            default: h.slot = 5, h.src = lin(a, b, 7), h.tx = a, h.ty = b, h.tz = -1, h.low = true; break;
        }
    } else {
        const int e = (hid - 384) >> 3, a = hid & 7;
        switch (e) {
            case 0: h.slot = 6, h.src = lin(7, 0, a), h.tx = -1, h.ty = 8, h.tz = a; break;
            case 1: h.slot = 7, h.src = lin(7, a, 0), h.tx = -1, h.ty = a, h.tz = 8; break;
            case 2: h.slot = 8, h.src = lin(0, 7, a), h.tx = 8, h.ty = -1, h.tz = a; break;
            case 3: h.slot = 9, h.src = lin(a, 7, 0), h.tx = a, h.ty = -1, h.tz = 8; break;
            case 4: h.slot = 10, h.src = lin(0, a, 7), h.tx = 8, h.ty = a, h.tz = -1; break;
            default: h.slot = 11, h.src = lin(a, 0, 7), h.tx = a, h.ty = 8, h.tz = -1; break;
        }
    }
    return h;
}

// Low-face voxel hd in [0, 192): faces -x, -y, -z.
__device__ inline void low_pos(int hd, int* x, int* y, int* z) {
    const int face = hd >> 6, a = hd & 7, b = (hd >> 3) & 7;
    if (face == 0) *x = -1, *y = a, *z = b;
    else if (face == 1) *x = a, *y = -1, *z = b;
    else *x = a, *y = b, *z = -1;
}

__device__ inline bool omega_bit(const uint32_t* __restrict__ bits, int block, int l) {
    return (__ldg(bits + (size_t)block * 16 + (l >> 5)) >> (l & 31)) & 1u;
}

struct Tiles {
    float v[kTile * kTile * kTile];             // u_bar (sweep) or u (energy)
    float p[3][kPTile * kPTile * kPTile];
    unsigned char om[kTile * kTile * kTile];
    int nb[kNeighbours];
};

// Stages the block's and its neighbours' values; thread t owns voxel t.
template <typename T>
__device__ inline void stage_tiles(Tiles& s, int b, const T* __restrict__ vsrc, const T* __restrict__ psrc,
                                   size_t pstride, const uint32_t* __restrict__ bits, const int32_t* __restrict__ nbr,
                                   int t, int lx, int ly, int lz, float& vc, bool& oc) {
    if (t < kNeighbours) s.nb[t] = __ldg(nbr + (size_t)b * kNeighbours + t);
    const size_t v = (size_t)b * kBlockVoxels + t;
    vc = Store<T>::ld(vsrc + v);
    oc = omega_bit(bits, b, t);
    s.v[t10(lx, ly, lz)] = vc;
    s.om[t10(lx, ly, lz)] = oc;
#pragma unroll
    for (int a = 0; a < 3; ++a) s.p[a][t9(lx, ly, lz)] = Store<T>::ld(psrc + a * pstride + v);
    __syncthreads();
    if (t < kHalo) {
        const HaloPos h = halo_pos(t);
        const int n = s.nb[h.slot];
        float hv = 0.0f, p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
        bool ho = false;
        if (n >= 0) {
            const size_t sv = (size_t)n * kBlockVoxels + h.src;
            hv = Store<T>::ld(vsrc + sv);
            ho = omega_bit(bits, n, h.src);
            if (h.low) {
                p0 = Store<T>::ld(psrc + sv);
                p1 = Store<T>::ld(psrc + pstride + sv);
                p2 = Store<T>::ld(psrc + 2 * pstride + sv);
            }
        }
        const int c = t10(h.tx, h.ty, h.tz);
        s.v[c] = hv;
        s.om[c] = ho;
        if (h.low) {
            const int q = t9(h.tx, h.ty, h.tz);
            s.p[0][q] = p0, s.p[1][q] = p1, s.p[2][q] = p2;
        }
    }
    __syncthreads();
}

// Arithmetic shared by every sweep variant, with explicit rounding so that all of
// them produce bit-identical iterates.
// Dual update of one voxel, Eq. 3: q = p + sigma grad; p' = q / max(1, |q|_2).  Inside
// the unit ball p' = q exactly; outside, q is scaled by the hardware reciprocal square
// root of |q|^2 (relative error below 2^-22).
__device__ inline void dual_update(float p0, float p1, float p2, float g0, float g1, float g2, float sigma,
                                   float* out) {
    const float q0 = __fmaf_rn(sigma, g0, p0);
    const float q1 = __fmaf_rn(sigma, g1, p1);
    const float q2 = __fmaf_rn(sigma, g2, p2);
    const float n2 = __fmaf_rn(q2, q2, __fmaf_rn(q1, q1, __fmul_rn(q0, q0)));
    const float sc = n2 > 1.0f ? rsqrtf(n2) : 1.0f;
    out[0] = __fmul_rn(q0, sc), out[1] = __fmul_rn(q1, sc), out[2] = __fmul_rn(q2, sc);
}

// Masked forward difference of Eq. 3.
__device__ inline float masked_diff(bool e, float next, float here) { return e ? __fsub_rn(next, here) : 0.0f; }

// Eq. 4 as the negative adjoint: own minus backward terms per axis, summed x, y, z.
__device__ inline float div_terms(bool ex, float px, bool exm, float pxm, bool ey, float py, bool eym, float pym,
                                  bool ez, float pz, bool ezm, float pzm) {
    const float d0 = __fsub_rn(ex ? px : 0.0f, exm ? pxm : 0.0f);
    const float d1 = __fsub_rn(ey ? py : 0.0f, eym ? pym : 0.0f);
    const float d2 = __fsub_rn(ez ? pz : 0.0f, ezm ? pzm : 0.0f);
    return __fadd_rn(__fadd_rn(d0, d1), d2);
}

// Primal proximal step on Omega and the relaxation (1 + tau lambda w >= 1: no denormal
// reaches the approximate reciprocal).
__device__ inline void primal_update(bool o, float uo, float dv, float fv, float wv, float tau, float tau_lam,
                                     float theta, float* un, float* ubn) {
    float u = uo;
    if (o) {
        const float ut = __fmaf_rn(tau, dv, uo);
        const float tlw = __fmul_rn(tau_lam, wv);
        u = __fmul_rn(__fmaf_rn(tlw, fv, ut), rcp_approx(__fadd_rn(1.0f, tlw)));
    }
    *un = u;
    *ubn = __fmaf_rn(theta, __fsub_rn(u, uo), u);
}

// Dual step at tile position (x, y, z): p <- P(p + sigma grad_Omega u_bar), Eq. 3.
__device__ inline void dual_step(Tiles& s, int x, int y, int z, float sigma, float* out) {
    const int c = t10(x, y, z);
    const bool o = s.om[c];
    const float u0 = s.v[c];
    const float g0 = masked_diff(o && s.om[c + 1], s.v[c + 1], u0);
    const float g1 = masked_diff(o && s.om[c + kTile], s.v[c + kTile], u0);
    const float g2 = masked_diff(o && s.om[c + kTile * kTile], s.v[c + kTile * kTile], u0);
    const int q = t9(x, y, z);
    dual_update(s.p[0][q], s.p[1][q], s.p[2][q], g0, g1, g2, sigma, out);
}

// Omega-aware divergence at a block voxel, Eq. 4 as the negative adjoint of Eq. 3.
__device__ inline float divergence(const Tiles& s, int x, int y, int z) {
    const int c = t10(x, y, z);
    const int q = t9(x, y, z);
    const bool o = s.om[c];
    return div_terms(o && s.om[c + 1], s.p[0][q], o && s.om[c - 1], s.p[0][q - 1], o && s.om[c + kTile], s.p[1][q],
                     o && s.om[c - kTile], s.p[1][q - kPTile], o && s.om[c + kTile * kTile], s.p[2][q],
                     o && s.om[c - kTile * kTile], s.p[2][q - kPTile * kPTile]);
}

template <typename T>
struct SweepArgs {
    const T* ub_in;
    T* ub_out;
    T* u;
    const T* p_in;
    T* p_out;
    const float* f;
    const float* w;
    const uint32_t* bits;
    const int32_t* nbr;
    const int32_t* order;  // visiting order of the blocks (NULL: index order)
    int32_t* err;          // sticky error flags (bounded waits that gave up)
    size_t pstride;
    int n_blocks;
    float sigma, tau, tau_lam, theta;
};

template <typename T>
__global__ void __launch_bounds__(kSweepThreads) sweep_kernel(SweepArgs<T> a) {
    __shared__ Tiles s;
    const int t = threadIdx.x;
    const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
    for (int b = blockIdx.x; b < a.n_blocks; b += gridDim.x) {
        float ubc;
        bool oc;
        stage_tiles<T>(s, b, a.ub_in, a.p_in, a.pstride, a.bits, a.nbr, t, lx, ly, lz, ubc, oc);
        const size_t v = (size_t)b * kBlockVoxels + t;
        const float uo = Store<T>::ld(a.u + v);
        const float fv = __ldg(a.f + v);
        const float wv = __ldg(a.w + v);
        float pc[3], ph[3];
        dual_step(s, lx, ly, lz, a.sigma, pc);
        int hx = 0, hy = 0, hz = 0;
        if (t < kLowHalo) {
            low_pos(t, &hx, &hy, &hz);
            dual_step(s, hx, hy, hz, a.sigma, ph);
        }
        __syncthreads();  // every read of the old p is done
        {
            const int q = t9(lx, ly, lz);
            s.p[0][q] = pc[0], s.p[1][q] = pc[1], s.p[2][q] = pc[2];
            if (t < kLowHalo) {
                const int qh = t9(hx, hy, hz);
                s.p[0][qh] = ph[0], s.p[1][qh] = ph[1], s.p[2][qh] = ph[2];
            }
        }
        __syncthreads();
        float un, ubn;
        primal_update(oc, uo, oc ? divergence(s, lx, ly, lz) : 0.0f, fv, wv, a.tau, a.tau_lam, a.theta, &un, &ubn);
        Store<T>::st(a.u + v, un);
        Store<T>::st(a.ub_out + v, ubn);
#pragma unroll
        for (int c = 0; c < 3; ++c) Store<T>::st(a.p_out + c * a.pstride + v, pc[c]);
        __syncthreads();  // the tiles are reused by the next block
    }
}

// ----------------------------------------------------------- pipelined sweep
// The same stencil as sweep_kernel, restructured for latency: a persistent CTA walks
// its blocks and, while it computes block k, cp.async copies already bring block k+1
// (core fields as 16-byte chunks, halo voxels and the neighbours' Omega words as
// 4-byte words) into the other half of a double-buffered shared-memory stage, and the
// neighbour row of block k+2 into a three-entry ring.  Block k's stage is then decoded
// into the padded float tiles the stencil functions read.
__device__ inline void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ inline void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// The same with zero fill: nothing is read and the destination is zeroed when !valid
// (src-size 0); gmem must still be a valid address.
__device__ inline void cp_async16z(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0) : "memory");
}
__device__ inline void cp_async4z(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Raw stage of one block (bytes; every part 16-byte aligned).
template <typename T>
struct StageLayout {
    static constexpr int E = (int)sizeof(T);
    static constexpr int kUb = 0;
    static constexpr int kP = kUb + kBlockVoxels * E;
    static constexpr int kU = kP + 3 * kBlockVoxels * E;
    static constexpr int kF = kU + kBlockVoxels * E;
    static constexpr int kW = kF + kBlockVoxels * 4;
    static constexpr int kBits = kW + kBlockVoxels * 4;
    static constexpr int kNBits = kBits + 64;
    static constexpr int kHaloUb = kNBits + kNeighbours * 64;
    static constexpr int kHaloP = kHaloUb + kHalo * 4;
    static constexpr int kBytes = kHaloP + 3 * kLowHalo * 4;
    // 16-byte chunks of the contiguous core part (u_bar, p, u, f, w, Omega bits)
    static constexpr int kCoreChunks = kNBits / 16;
};

// Low-face index (0..191) of halo entry hid, or -1.
__device__ inline int low_index(int hid) {
    if (hid >= 64 && hid < 128) return hid - 64;
    if (hid >= 192 && hid < 256) return hid - 192 + 64;
    if (hid >= 320 && hid < 384) return hid - 320 + 128;
    return -1;
}
__device__ inline int low_hid(int li) { return li < 64 ? li + 64 : (li < 128 ? li - 64 + 192 : li - 128 + 320); }

// Element e of a 4-byte word that holds element offset `off` of a T array.
template <typename T>
__device__ inline float word_elem(uint32_t w, int off) {
    if constexpr (sizeof(T) == 4) {
        return __uint_as_float(w);
    } else {
        const unsigned short h = (off & 1) ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xffffu);
        T v;
        memcpy(&v, &h, 2);
        return Store<T>::ld(&v);
    }
}

template <typename T>
__device__ inline const void* word_addr(const T* base, size_t off) {
    return reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(base + off) & ~(uintptr_t)3);
}

// Issues the copies of block b's core and its neighbour row (for the ring).
template <typename T>
__device__ inline void issue_core(const SweepArgs<T>& a, char* st, int b, int* nbr_slot_next, int b_next, int t) {
    using L = StageLayout<T>;
    const size_t v0 = (size_t)b * kBlockVoxels;
    for (int c = t; c < L::kCoreChunks; c += kSweepThreads) {
        const int off = c * 16;
        const char* src;
        if (off < L::kP) src = reinterpret_cast<const char*>(a.ub_in + v0) + off;
        else if (off < L::kU) {
            const int q = off - L::kP, comp = q / (kBlockVoxels * L::E);
            src = reinterpret_cast<const char*>(a.p_in + comp * a.pstride + v0) + (q - comp * kBlockVoxels * L::E);
        } else if (off < L::kF) src = reinterpret_cast<const char*>(a.u + v0) + (off - L::kU);
        else if (off < L::kW) src = reinterpret_cast<const char*>(a.f + v0) + (off - L::kF);
        else if (off < L::kBits) src = reinterpret_cast<const char*>(a.w + v0) + (off - L::kW);
        else src = reinterpret_cast<const char*>(a.bits + (size_t)b * 16) + (off - L::kBits);
        cp_async16(st + off, src);
    }
    if (b_next >= 0 && t < 3) cp_async16(nbr_slot_next + 4 * t, a.nbr + (size_t)b_next * kNeighbours + 4 * t);
}

// Issues the halo copies of block b (needs its neighbour row in shared memory).
template <typename T>
__device__ inline void issue_halo(const SweepArgs<T>& a, char* st, const int* nb, int t) {
    using L = StageLayout<T>;
    if (t < kHalo) {
        const HaloPos h = halo_pos(t);
        const int n = nb[h.slot];
        if (n >= 0) cp_async4(st + L::kHaloUb + 4 * t, word_addr(a.ub_in, (size_t)n * kBlockVoxels + h.src));
    }
    for (int i = t; i < 3 * kLowHalo; i += kSweepThreads) {
        const int comp = i / kLowHalo, li = i - comp * kLowHalo;
        const HaloPos h = halo_pos(low_hid(li));
        const int n = nb[h.slot];
        if (n >= 0)
            cp_async4(st + L::kHaloP + 4 * i, word_addr(a.p_in + comp * a.pstride, (size_t)n * kBlockVoxels + h.src));
    }
    if (t < kNeighbours * 4) {
        const int e = t >> 2, q = t & 3;
        const int n = nb[e];
        if (n >= 0) cp_async16(st + L::kNBits + 64 * e + 16 * q, a.bits + (size_t)n * 16 + 4 * q);
    }
}

// Decodes a completed stage into the stencil tiles; returns the core voxel's values.
template <typename T>
__device__ inline void decode_stage(Tiles& s, const char* st, const int* nb, int t, int lx, int ly, int lz, bool& oc) {
    using L = StageLayout<T>;
    const T* cub = reinterpret_cast<const T*>(st + L::kUb);
    const T* cp = reinterpret_cast<const T*>(st + L::kP);
    const uint32_t* bits = reinterpret_cast<const uint32_t*>(st + L::kBits);
    oc = (bits[t >> 5] >> (t & 31)) & 1u;
    const int c = t10(lx, ly, lz), q = t9(lx, ly, lz);
    s.v[c] = Store<T>::ld(cub + t);
    s.om[c] = oc;
#pragma unroll
    for (int k = 0; k < 3; ++k) s.p[k][q] = Store<T>::ld(cp + k * kBlockVoxels + t);
    if (t < kHalo) {
        const HaloPos h = halo_pos(t);
        const int n = nb[h.slot];
        const int hc = t10(h.tx, h.ty, h.tz);
        float hv = 0.0f;
        bool ho = false;
        if (n >= 0) {
            hv = word_elem<T>(reinterpret_cast<const uint32_t*>(st + L::kHaloUb)[t], h.src);
            const uint32_t* nbits = reinterpret_cast<const uint32_t*>(st + L::kNBits) + 16 * h.slot;
            ho = (nbits[h.src >> 5] >> (h.src & 31)) & 1u;
        }
        s.v[hc] = hv;
        s.om[hc] = ho;
        const int li = low_index(t);
        if (li >= 0) {
            const int hq = t9(h.tx, h.ty, h.tz);
            const uint32_t* hp = reinterpret_cast<const uint32_t*>(st + L::kHaloP);
#pragma unroll
            for (int k = 0; k < 3; ++k) s.p[k][hq] = n >= 0 ? word_elem<T>(hp[k * kLowHalo + li], h.src) : 0.0f;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kSweepThreads, 2) sweep_pipe_kernel(SweepArgs<T> a) {
    using L = StageLayout<T>;
    extern __shared__ __align__(16) char smem[];
    Tiles& s = *reinterpret_cast<Tiles*>(smem);
    char* stage0 = smem + ((sizeof(Tiles) + 15) / 16) * 16;
    int* ring = reinterpret_cast<int*>(stage0 + 2 * L::kBytes);  // [3][12]
    const int t = threadIdx.x;
    const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
    const int G = gridDim.x;
    int b = blockIdx.x;
    if (b >= a.n_blocks) return;
    auto block_at = [&](int k) -> int {
        const int i = blockIdx.x + k * G;
        return i < a.n_blocks ? (a.order ? __ldg(a.order + i) : i) : -1;
    };
    int b_cur = block_at(0);
    // prologue: neighbour row of the first block, then its core and halos
    if (t < kNeighbours) ring[t] = __ldg(a.nbr + (size_t)b_cur * kNeighbours + t);
    __syncthreads();
    issue_core<T>(a, stage0, b_cur, ring + kNeighbours, block_at(1), t);
    issue_halo<T>(a, stage0, ring, t);
    cp_async_commit();
    for (int k = 0; b_cur >= 0; ++k) {
        char* st = stage0 + (k & 1) * L::kBytes;
        const int* nb = ring + (k % 3) * kNeighbours;
        cp_async_wait_all();
        __syncthreads();
        const int b_next = block_at(k + 1);
        if (b_next >= 0) {
            char* st2 = stage0 + ((k + 1) & 1) * L::kBytes;
            issue_core<T>(a, st2, b_next, ring + ((k + 2) % 3) * kNeighbours, block_at(k + 2), t);
            issue_halo<T>(a, st2, ring + ((k + 1) % 3) * kNeighbours, t);
            cp_async_commit();
        }
        bool oc;
        decode_stage<T>(s, st, nb, t, lx, ly, lz, oc);
        const float uo = Store<T>::ld(reinterpret_cast<const T*>(st + L::kU) + t);
        const float fv = reinterpret_cast<const float*>(st + L::kF)[t];
        const float wv = reinterpret_cast<const float*>(st + L::kW)[t];
        __syncthreads();
        float pc[3], ph[3];
        dual_step(s, lx, ly, lz, a.sigma, pc);
        int hx = 0, hy = 0, hz = 0;
        if (t < kLowHalo) {
            low_pos(t, &hx, &hy, &hz);
            dual_step(s, hx, hy, hz, a.sigma, ph);
        }
        __syncthreads();
        {
            const int q = t9(lx, ly, lz);
            s.p[0][q] = pc[0], s.p[1][q] = pc[1], s.p[2][q] = pc[2];
            if (t < kLowHalo) {
                const int qh = t9(hx, hy, hz);
                s.p[0][qh] = ph[0], s.p[1][qh] = ph[1], s.p[2][qh] = ph[2];
            }
        }
        __syncthreads();
        float un, ubn;
        primal_update(oc, uo, oc ? divergence(s, lx, ly, lz) : 0.0f, fv, wv, a.tau, a.tau_lam, a.theta, &un, &ubn);
        const size_t v = (size_t)b_cur * kBlockVoxels + t;
        Store<T>::st(a.u + v, un);
        Store<T>::st(a.ub_out + v, ubn);
#pragma unroll
        for (int c = 0; c < 3; ++c) Store<T>::st(a.p_out + c * a.pstride + v, pc[c]);
        b_cur = b_next;
    }
}

// --------------------------------------------------------------- row sweep
// One 64-thread CTA per block at a time (grid-stride over the visiting order); thread
// r owns the x-row (ly, lz) = (r & 7, r >> 3), i.e. 8 consecutive voxels that move as
// 16-byte vectors.  x-neighbours stay in registers; only the y/z-neighbour rows and the
// block faces pass through shared memory.  Every thread also takes the dual step at
// the voxel just behind its row (the -x face), and the threads on the low y and z
// faces take it on the neighbour rows behind them, because the divergence reads
// p^{k+1} one voxel behind the block.
constexpr int kRowThreads = 64;

__device__ inline int r10(int ly, int lz) { return (ly + 1) + 10 * (lz + 1); }
__device__ inline int r9(int ly, int lz) { return (ly + 1) + 9 * (lz + 1); }

struct __align__(16) RowTiles {
    float ub[100][8];        // u_bar rows (ly, lz) in [-1, 8]^2
    float py[81][8];         // new p_y on rows (ly, lz) in [-1, 7]^2
    float pz[81][8];         // new p_z
    float pfy[3][8][8];      // old p on the -y face rows (-1, lz)
    float pfz[3][8][8];      // old p on the -z face rows (ly, -1)
    float xhp[100];          // u_bar at x = 8 of each row
    float xhm[100];          // u_bar at x = -1 of each row
    float pxm[64];           // new p_x at x = -1 of each block row
    float phm[3][64];        // old p at x = -1 of each block row (asynchronous staging)
    unsigned short om[100];  // Omega: bits 0-7 at x = 0..7, bit 8 at x = 8, bit 9 at x = -1
};

// 8 stored 16-bit values (one 16-byte word) as floats, converted in pairs.
template <typename T>
__device__ inline void unpack8(const uint4& q, float* v) {
    const float2 a = Store<T>::ld2(q.x), b = Store<T>::ld2(q.y), c = Store<T>::ld2(q.z), d = Store<T>::ld2(q.w);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y, v[4] = c.x, v[5] = c.y, v[6] = d.x, v[7] = d.y;
}

template <typename T>
__device__ inline void ld_row(const T* __restrict__ p, float* v) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    } else {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
        unpack8<T>(q, v);
    }
}

template <typename T>
__device__ inline void st_row(T* p, const float* v) {
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
        *reinterpret_cast<uint4*>(p) = make_uint4(Store<T>::st2(v[0], v[1]), Store<T>::st2(v[2], v[3]),
                                                  Store<T>::st2(v[4], v[5]), Store<T>::st2(v[6], v[7]));
    }
}

__device__ inline void sts_row(float* dst, const float* v) {
    reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

__device__ inline void lds_row(const float* src, float* v) {
    const float4 a = reinterpret_cast<const float4*>(src)[0];
    const float4 b = reinterpret_cast<const float4*>(src)[1];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}

// Omega bits of x-row `row` of block n (x = 0..7) in the low byte.
__device__ inline unsigned row_bits(const uint32_t* __restrict__ bits, int n, int row) {
    return (__ldg(bits + (size_t)n * 16 + (row >> 2)) >> (8 * (row & 3))) & 0xffu;
}

// Loads a full neighbour row (x = 0..7) of block n into tile row `dst` with its Omega
// byte; zeros (Omega-bar) when the block is not allocated.
template <typename T>
__device__ inline unsigned load_face_row(const SweepArgs<T>& a, int n, int src_row, float* dst) {
    float v[8];
    unsigned om = 0;
    if (n >= 0) {
        ld_row<T>(a.ub_in + (size_t)n * kBlockVoxels + 8 * src_row, v);
        om = row_bits(a.bits, n, src_row);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.0f;
    }
    sts_row(dst, v);
    return om;
}

// One voxel of a neighbour block (u_bar value and Omega bit at offset l).
template <typename T>
__device__ inline float load_voxel(const SweepArgs<T>& a, int n, int l, unsigned* bit) {
    if (n < 0) {
        *bit = 0;
        return 0.0f;
    }
    *bit = (__ldg(a.bits + (size_t)n * 16 + (l >> 5)) >> (l & 31)) & 1u;
    return Store<T>::ld(a.ub_in + (size_t)n * kBlockVoxels + l);
}

// Shared-memory stage of one block's own fields, filled by 1-D bulk copies (TMA).
template <typename T>
struct RowStage {
    static constexpr int kField = kBlockVoxels * (int)sizeof(T);
    static constexpr int kUb = 0;
    static constexpr int kP = kUb + kField;
    static constexpr int kU = kP + 3 * kField;
    static constexpr int kF = kU + kField;
    static constexpr int kW = kF + kBlockVoxels * 4;
    static constexpr int kBits = kW + kBlockVoxels * 4;
    static constexpr int kTx = kBits + 64;                 // bytes the copies deliver
    static constexpr int kBytes = (kTx + 127) / 128 * 128;  // stride between the two stages
};

template <typename T>
__device__ inline void ld_row_smem(const T* p, float* v) {
    if constexpr (sizeof(T) == 4) {
        lds_row(reinterpret_cast<const float*>(p), v);
    } else {
        unpack8<T>(*reinterpret_cast<const uint4*>(p), v);
    }
}

// Where the asynchronous halo copies land.  With float32 storage they land in the tiles
// themselves.  With 16-bit storage they land here first, as stored (a row of 8 values;
// for a single voxel the aligned 4-byte word that holds it, since cp.async moves at least
// 4 bytes), and each thread converts what it copied into the tiles.
template <typename T>
struct __align__(16) HaloRaw {
    T ub[100][8];
    T pfy[3][8][8];
    T pfz[3][8][8];
    uint32_t xhp[100], xhm[100];
    uint32_t phm[3][64];
};
template <>
struct HaloRaw<float> {
    int unused;
};

// Row `row` of block n's field (8 values: 32 or 16 bytes); zeros when n < 0.
template <typename T>
__device__ inline void cp_row_z(void* dst, const T* field, int n, int row) {
    const bool ok = n >= 0;
    const T* src = ok ? field + (size_t)n * kBlockVoxels + 8 * row : field;
    cp_async16z(dst, src, ok);
    if constexpr (sizeof(T) == 4) cp_async16z(reinterpret_cast<char*>(dst) + 16, ok ? src + 4 : field, ok);
}

// Voxel l of block n's field (16-bit storage: the 4-byte word holding it); zero when n < 0.
template <typename T>
__device__ inline void cp_voxel_z(void* dst, const T* field, int n, int l) {
    const int la = sizeof(T) == 4 ? l : (l & ~1);
    cp_async4z(dst, n >= 0 ? field + (size_t)n * kBlockVoxels + la : field, n >= 0);
}

__device__ inline unsigned voxel_bit(const uint32_t* __restrict__ bits, int n, int l) {
    return n >= 0 ? (__ldg(bits + (size_t)n * 16 + (l >> 5)) >> (l & 31)) & 1u : 0u;
}

// The value of a 16-bit voxel from the word that holds it (odd: the upper half).
template <typename T>
__device__ inline float word_half(uint32_t w, int odd) {
    return Store<T>::ld(reinterpret_cast<const T*>(&w) + odd);
}

// Balanced face staging.  Besides the x halos of its own rows, a block's stencil reads
// 34 u_bar rows of its neighbours (8 behind each of the four y and z faces, and the two
// edge rows the -y and -z face voxels' dual steps read), the 32 voxels at the x ends of
// the four face rows and 48 rows of old p behind the -y and -z faces.  They are split
// into 82 row items:
//   0-31   u_bar face row j of face F (F = i / 8: +y, -y, +z, -z), with its end voxel
//          and the tile row's Omega word;
//   32-79  p row: k = i - 32, component (k % 24) / 8 of row k % 8 behind -y (k < 24)
//          or -z (the pfy and pfz tiles read as one array of 48 rows);
//   80-81  the edge rows (-1, 8) and (8, -1).
// Thread t takes item t and, for t < 18, item t + 64, so each warp runs one or two kinds
// of item with most lanes active instead of one branch per face with four or eight.
struct FaceRow {
    int n, row, d;     // source block, source row, tile row
    int ne, le, odd;   // end voxel: source block, offset; odd: at x = -1 (else x = 8)
};

__device__ __forceinline__ FaceRow face_row(const int* nb, int i) {
    const int F = i >> 3, j = i & 7;
    FaceRow f;
    f.n = F == 0 ? nb[1] : (F == 1 ? nb[4] : (F == 2 ? nb[2] : nb[5]));
    f.ne = F == 0 ? nb[6] : (F == 1 ? nb[8] : (F == 2 ? nb[7] : nb[10]));
    // +y: tile row (8, j) <- row (0, j), end voxel (-1, 8, j) <- (7, 0, j) of block (-x,+y)
    // -y: tile row (-1, j) <- row (7, j), end voxel (8, -1, j) <- (0, 7, j) of block (+x,-y)
    // +z: tile row (j, 8) <- row (j, 0), end voxel (-1, j, 8) <- (7, j, 0) of block (-x,+z)
    // -z: tile row (j, -1) <- row (j, 7), end voxel (8, j, -1) <- (0, j, 7) of block (+x,-z)
    f.row = F == 0 ? 8 * j : (F == 1 ? 7 + 8 * j : (F == 2 ? j : 56 + j));
    f.d = F == 0 ? 19 + 10 * j : (F == 1 ? 10 + 10 * j : (F == 2 ? 91 + j : 1 + j));
    f.odd = (F & 1) ^ 1;
    f.le = 8 * f.row + (f.odd ? 7 : 0);
    return f;
}

// p item k in [0, 48): source block, source row and component.
__device__ __forceinline__ void p_row_item(const int* nb, int k, int* n, int* row, int* c) {
    const bool zf = k >= 24;
    const int kk = zf ? k - 24 : k, j = kk & 7;
    *c = kk >> 3;
    *n = zf ? nb[5] : nb[4];
    *row = zf ? 56 + j : 7 + 8 * j;
}

// Issues the copies of the balanced face items of thread t (cp.async, zero fill), and
// stores the Omega words of the tile rows they fill.
template <typename T>
__device__ __forceinline__ void issue_faces_balanced(const SweepArgs<T>& a, RowTiles& s, HaloRaw<T>& raw, int t,
                                                     const int* nb) {
    constexpr bool kF = sizeof(T) == 4;
    static_assert(offsetof(RowTiles, pfz) == offsetof(RowTiles, pfy) + sizeof(float) * 192, "pfy/pfz layout");
    auto ub_row = [&](int d) -> void* { if constexpr (kF) return s.ub[d]; else return raw.ub[d]; };
    auto p_dst = [&](int k) -> void* {
        if constexpr (kF) return &s.pfy[0][0][0] + 8 * k; else return &raw.pfy[0][0][0] + 8 * k;
    };
    if (t < 32) {
        const FaceRow f = face_row(nb, t);
        cp_row_z<T>(ub_row(f.d), a.ub_in, f.n, f.row);
        void* xd;
        if constexpr (kF) xd = f.odd ? &s.xhm[f.d] : &s.xhp[f.d]; else xd = f.odd ? &raw.xhm[f.d] : &raw.xhp[f.d];
        cp_voxel_z<T>(xd, a.ub_in, f.ne, f.le);
        s.om[f.d] = (unsigned short)((f.n >= 0 ? row_bits(a.bits, f.n, f.row) : 0u) |
                                     (voxel_bit(a.bits, f.ne, f.le) << (f.odd ? 9 : 8)));
    } else {
        int n, row, c;
        p_row_item(nb, t - 32, &n, &row, &c);
        cp_row_z<T>(p_dst(t - 32), a.p_in + c * a.pstride, n, row);
    }
    if (t < 16) {
        int n, row, c;
        p_row_item(nb, t + 32, &n, &row, &c);
        cp_row_z<T>(p_dst(t + 32), a.p_in + c * a.pstride, n, row);
    } else if (t < 18) {
        const int n = t == 16 ? nb[9] : nb[11], row = t == 16 ? 7 : 56, d = t == 16 ? 90 : 9;
        cp_row_z<T>(ub_row(d), a.ub_in, n, row);
        s.om[d] = (unsigned short)(n >= 0 ? row_bits(a.bits, n, row) : 0u);
    }
}

// 16-bit storage: converts what issue_faces_balanced copied for thread t (after its
// copies have landed) into the float32 tiles.
template <typename T>
__device__ __forceinline__ void convert_faces_balanced(RowTiles& s, const HaloRaw<T>& raw, int t, const int* nb) {
    static_assert(offsetof(HaloRaw<T>, pfz) == offsetof(HaloRaw<T>, pfy) + sizeof(T) * 192, "pfy/pfz layout");
    auto row = [&](float* dst, const T* src) {
        float v[8];
        unpack8<T>(*reinterpret_cast<const uint4*>(src), v);
        sts_row(dst, v);
    };
    if (t < 32) {
        const FaceRow f = face_row(nb, t);
        row(s.ub[f.d], raw.ub[f.d]);
        if (f.odd) s.xhm[f.d] = word_half<T>(raw.xhm[f.d], 1);
        else s.xhp[f.d] = word_half<T>(raw.xhp[f.d], 0);
    } else {
        row(&s.pfy[0][0][0] + 8 * (t - 32), &raw.pfy[0][0][0] + 8 * (t - 32));
    }
    if (t < 16) row(&s.pfy[0][0][0] + 8 * (t + 32), &raw.pfy[0][0][0] + 8 * (t + 32));
    else if (t < 18) row(s.ub[t == 16 ? 90 : 9], raw.ub[t == 16 ? 90 : 9]);
}

// 16-bit storage with balanced face items: converts the x halos of row r and thread r's
// face items (after their copies have landed) into the float32 tiles.
template <typename T>
__device__ __forceinline__ void convert_halos_balanced(RowTiles& s, const HaloRaw<T>& raw, int r, int ly, int lz,
                                                       const int* nb) {
    const int rr = r10(ly, lz);
    s.xhp[rr] = word_half<T>(raw.xhp[rr], 0);
    s.xhm[rr] = word_half<T>(raw.xhm[rr], 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) s.phm[c][r] = word_half<T>(raw.phm[c][r], 1);
    convert_faces_balanced<T>(s, raw, r, nb);
}

// The same items loaded synchronously (through registers) into the float32 tiles.
template <typename T>
__device__ __forceinline__ void load_faces_balanced(const SweepArgs<T>& a, RowTiles& s, int t, const int* nb) {
    auto p_row = [&](int k) {
        int n, row, c;
        p_row_item(nb, k, &n, &row, &c);
        float q[8];
        if (n >= 0) {
            ld_row<T>(a.p_in + c * a.pstride + (size_t)n * kBlockVoxels + 8 * row, q);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = 0.0f;
        }
        sts_row(&s.pfy[0][0][0] + 8 * k, q);
    };
    if (t < 32) {
        const FaceRow f = face_row(nb, t);
        const unsigned om = load_face_row<T>(a, f.n, f.row, s.ub[f.d]);
        unsigned bit;
        const float v = load_voxel<T>(a, f.ne, f.le, &bit);
        if (f.odd) s.xhm[f.d] = v;
        else s.xhp[f.d] = v;
        s.om[f.d] = (unsigned short)(om | (bit << (f.odd ? 9 : 8)));
    } else {
        p_row(t - 32);
    }
    if (t < 16) {
        p_row(t + 32);
    } else if (t < 18) {
        const int d = t == 16 ? 90 : 9;
        s.om[d] = (unsigned short)load_face_row<T>(a, t == 16 ? nb[9] : nb[11], t == 16 ? 7 : 56, s.ub[d]);
    }
}

// Asynchronous halo staging of row r: the x halos, the face and edge rows and the old p
// behind the low faces go straight from L2 into shared memory (cp.async, zeros for
// absent neighbours), so that their latency overlaps the loads of the block's own rows.
// Returns the Omega words of the tile rows the row fills: om[0] the x-halo bits of its
// own row (bits 8 and 9), om[1] its y-face row, om[2] its z-face row, om[3] its edge row.
// The x = 8 voxels sit at even offsets of their block, the x = -1 voxels at odd ones.
template <typename T, bool BAL = false>
__device__ __forceinline__ void issue_row_halos(const SweepArgs<T>& a, RowTiles& s, HaloRaw<T>& raw, int r, int ly,
                                                int lz, const int* nb, unsigned* om) {
    constexpr bool kF = sizeof(T) == 4;
    const T* ubs = a.ub_in;
    const size_t ps = a.pstride;
    const int rr = r10(ly, lz);
    auto ub_row = [&](int d) -> void* { if constexpr (kF) return s.ub[d]; else return raw.ub[d]; };
    auto xhp = [&](int d) -> void* { if constexpr (kF) return &s.xhp[d]; else return &raw.xhp[d]; };
    auto xhm = [&](int d) -> void* { if constexpr (kF) return &s.xhm[d]; else return &raw.xhm[d]; };
    cp_voxel_z<T>(xhp(rr), ubs, nb[0], 8 * r);
    cp_voxel_z<T>(xhm(rr), ubs, nb[3], 8 * r + 7);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        void* dst;
        if constexpr (kF) dst = &s.phm[c][r]; else dst = &raw.phm[c][r];
        cp_voxel_z<T>(dst, a.p_in + c * ps, nb[3], 8 * r + 7);
    }
    om[0] = (voxel_bit(a.bits, nb[0], 8 * r) << 8) | (voxel_bit(a.bits, nb[3], 8 * r + 7) << 9);
    om[1] = om[2] = om[3] = 0u;
    if constexpr (BAL) {
        issue_faces_balanced<T>(a, s, raw, r, nb);
        cp_async_commit();
        return;
    }
    if (ly == 7) {  // row (8, lz) <- block +y row (0, lz); edge (-1, 8, lz) <- block (-x,+y) voxel (7, 0, lz)
        const int d = r10(8, lz);
        cp_row_z<T>(ub_row(d), ubs, nb[1], 8 * lz);
        cp_voxel_z<T>(xhm(d), ubs, nb[6], 8 * (8 * lz) + 7);
        om[1] = (nb[1] >= 0 ? row_bits(a.bits, nb[1], 8 * lz) : 0u) | (voxel_bit(a.bits, nb[6], 8 * (8 * lz) + 7) << 9);
    }
    if (ly == 0) {  // row (-1, lz) <- block -y row (7, lz); edge (8, -1, lz) <- block (-y,+x) voxel (0, 7, lz)
        const int d = r10(-1, lz);
        cp_row_z<T>(ub_row(d), ubs, nb[4], 7 + 8 * lz);
        cp_voxel_z<T>(xhp(d), ubs, nb[8], 8 * (7 + 8 * lz));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            void* dst;
            if constexpr (kF) dst = s.pfy[c][lz]; else dst = raw.pfy[c][lz];
            cp_row_z<T>(dst, a.p_in + c * ps, nb[4], 7 + 8 * lz);
        }
        om[1] = (nb[4] >= 0 ? row_bits(a.bits, nb[4], 7 + 8 * lz) : 0u) | (voxel_bit(a.bits, nb[8], 8 * (7 + 8 * lz)) << 8);
    }
    if (lz == 7) {  // row (ly, 8) <- block +z row (ly, 0); edge (-1, ly, 8) <- block (-x,+z) voxel (7, ly, 0)
        const int d = r10(ly, 8);
        cp_row_z<T>(ub_row(d), ubs, nb[2], ly);
        cp_voxel_z<T>(xhm(d), ubs, nb[7], 8 * ly + 7);
        om[2] = (nb[2] >= 0 ? row_bits(a.bits, nb[2], ly) : 0u) | (voxel_bit(a.bits, nb[7], 8 * ly + 7) << 9);
    }
    if (lz == 0) {  // row (ly, -1) <- block -z row (ly, 7); edge (8, ly, -1) <- block (-z,+x) voxel (0, ly, 7)
        const int d = r10(ly, -1);
        cp_row_z<T>(ub_row(d), ubs, nb[5], ly + 56);
        cp_voxel_z<T>(xhp(d), ubs, nb[10], 8 * (ly + 56));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            void* dst;
            if constexpr (kF) dst = s.pfz[c][ly]; else dst = raw.pfz[c][ly];
            cp_row_z<T>(dst, a.p_in + c * ps, nb[5], ly + 56);
        }
        om[2] = (nb[5] >= 0 ? row_bits(a.bits, nb[5], ly + 56) : 0u) | (voxel_bit(a.bits, nb[10], 8 * (ly + 56)) << 8);
    }
    if (ly == 0 && lz == 7) {  // edge row (-1, 8) <- block (-y,+z) row (7, 0)
        cp_row_z<T>(ub_row(r10(-1, 8)), ubs, nb[9], 7);
        om[3] = nb[9] >= 0 ? row_bits(a.bits, nb[9], 7) : 0u;
    }
    if (ly == 7 && lz == 0) {  // edge row (8, -1) <- block (-z,+y) row (0, 7)
        cp_row_z<T>(ub_row(r10(8, -1)), ubs, nb[11], 56);
        om[3] = nb[11] >= 0 ? row_bits(a.bits, nb[11], 56) : 0u;
    }
    cp_async_commit();
}

// 16-bit storage: converts the halo values row r copied (after its copies have landed)
// into the float32 tiles.
template <typename T>
__device__ __forceinline__ void convert_row_halos(RowTiles& s, const HaloRaw<T>& raw, int r, int ly, int lz) {
    const int rr = r10(ly, lz);
    auto row = [&](float* dst, const T* src) {
        float v[8];
        unpack8<T>(*reinterpret_cast<const uint4*>(src), v);
        sts_row(dst, v);
    };
    s.xhp[rr] = word_half<T>(raw.xhp[rr], 0);
    s.xhm[rr] = word_half<T>(raw.xhm[rr], 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) s.phm[c][r] = word_half<T>(raw.phm[c][r], 1);
    if (ly == 7) {
        const int d = r10(8, lz);
        row(s.ub[d], raw.ub[d]);
        s.xhm[d] = word_half<T>(raw.xhm[d], 1);
    }
    if (ly == 0) {
        const int d = r10(-1, lz);
        row(s.ub[d], raw.ub[d]);
        s.xhp[d] = word_half<T>(raw.xhp[d], 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) row(s.pfy[c][lz], raw.pfy[c][lz]);
    }
    if (lz == 7) {
        const int d = r10(ly, 8);
        row(s.ub[d], raw.ub[d]);
        s.xhm[d] = word_half<T>(raw.xhm[d], 1);
    }
    if (lz == 0) {
        const int d = r10(ly, -1);
        row(s.ub[d], raw.ub[d]);
        s.xhp[d] = word_half<T>(raw.xhp[d], 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) row(s.pfz[c][ly], raw.pfz[c][ly]);
    }
    if (ly == 0 && lz == 7) row(s.ub[r10(-1, 8)], raw.ub[r10(-1, 8)]);
    if (ly == 7 && lz == 0) row(s.ub[r10(8, -1)], raw.ub[r10(8, -1)]);
}

// Per-thread stage of the prefetching row sweep: thread r's slot holds row r of the
// next block's own fields (u_bar, p_x, p_y, p_z, u as stored, f, w as float32) and the
// Omega word that holds the row's bits.  Each thread copies and later reads only its own
// slot, so the stage needs no barrier.  The slot strides (240 and 176 bytes, 60 and 44
// words) put the 16-byte reads of eight consecutive threads on distinct banks.
template <typename T>
struct OwnSlot {
    static constexpr int kRowT = 8 * (int)sizeof(T);
    static constexpr int kUb = 0;
    static constexpr int kP = kRowT;
    static constexpr int kU = 4 * kRowT;
    static constexpr int kF = 5 * kRowT;
    static constexpr int kW = kF + 32;
    static constexpr int kBits = kW + 32;
    static constexpr int kBytes = sizeof(T) == 4 ? 240 : 176;
    static_assert(kBits + 4 <= kBytes, "slot too small");
};

// 8 values of a stored field (32 or 16 bytes) by cp.async into a slot.
template <typename T>
__device__ inline void cp_row(char* dst, const T* src) {
    cp_async16(dst, src);
    if constexpr (sizeof(T) == 4) cp_async16(dst + 16, src + 4);
}

// Issues the copies of row r of block b's own fields into the thread's slot.
template <typename T>
__device__ __forceinline__ void issue_own_row(const SweepArgs<T>& a, char* slot, int b, int r) {
    using L = OwnSlot<T>;
    const size_t base = (size_t)b * kBlockVoxels + 8 * r;
    cp_row<T>(slot + L::kUb, a.ub_in + base);
#pragma unroll
    for (int c = 0; c < 3; ++c) cp_row<T>(slot + L::kP + c * L::kRowT, a.p_in + c * a.pstride + base);
    cp_row<T>(slot + L::kU, a.u + base);
    cp_row<float>(slot + L::kF, a.f + base);
    cp_row<float>(slot + L::kW, a.w + base);
    cp_async4(slot + L::kBits, a.bits + (size_t)b * 16 + (r >> 2));
}

// The arithmetic half of one block of the row sweep, after its staging: the dual steps
// (the row's voxels, its -x voxel and one voxel of each low face), then the primal step
// and the relaxation, and the stores.  om_r holds the row's Omega bits (0-7) and those of
// its x halos (8: x = 8, 9: x = -1); hm0..hm2 the old p at x = -1.
template <typename T>
__device__ __forceinline__ void rows_compute(const SweepArgs<T>& a, RowTiles& s, int r, unsigned om_r, float* ub,
                                             float* p0, float* p1, float* p2, const float* uo, const float* fv,
                                             const float* wv, float hm0, float hm1, float hm2, size_t base) {
    const int ly = r & 7, lz = r >> 3;
    const int rr = r10(ly, lz);
    const size_t ps = a.pstride;
    // ------------------------------------------------------- dual steps
    {
        float uy[8], uz[8];
        lds_row(s.ub[r10(ly + 1, lz)], uy);
        lds_row(s.ub[r10(ly, lz + 1)], uz);
        const unsigned om_y = s.om[r10(ly + 1, lz)], om_z = s.om[r10(ly, lz + 1)];
        const float xp = s.xhp[rr];
        // Eq. 3 edge masks of the row, one bit per voxel (bit 8 of om_r is the +x halo)
        const unsigned ex = om_r & (om_r >> 1), ey = om_r & om_y, ez = om_r & om_z;
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const float g0 = masked_diff((ex >> x) & 1u, x < 7 ? ub[x < 7 ? x + 1 : 7] : xp, ub[x]);
            const float g1 = masked_diff((ey >> x) & 1u, uy[x], ub[x]);
            const float g2 = masked_diff((ez >> x) & 1u, uz[x], ub[x]);
            float out[3];
            dual_update(p0[x], p1[x], p2[x], g0, g1, g2, a.sigma, out);
            p0[x] = out[0], p1[x] = out[1], p2[x] = out[2];
        }
        // the -x face voxel (-1, ly, lz)
        const bool o = (om_r >> 9) & 1u;
        const float um = s.xhm[rr];
        const int ry = r10(ly + 1, lz), rz = r10(ly, lz + 1);
        const float g0 = masked_diff(o && (om_r & 1u), ub[0], um);
        const float g1 = masked_diff(o && ((s.om[ry] >> 9) & 1u), s.xhm[ry], um);
        const float g2 = masked_diff(o && ((s.om[rz] >> 9) & 1u), s.xhm[rz], um);
        float out[3];
        dual_update(hm0, hm1, hm2, g0, g1, g2, a.sigma, out);
        s.pxm[r] = out[0];
    }
    {
        // one voxel of the -y face, (fx, -1, fz), and one of the -z face, (fx, fy, -1)
        const int fx = r & 7, fw = r >> 3;
        {  // -y face: fw is z
            const int d = r10(-1, fw), dz = r10(-1, fw + 1), dc = r10(0, fw);
            const unsigned om = s.om[d];
            const bool o = (om >> fx) & 1u;
            const float v = s.ub[d][fx];
            const float g0 = masked_diff(o && ((om >> (fx + 1)) & 1u), fx < 7 ? s.ub[d][fx < 7 ? fx + 1 : 7] : s.xhp[d], v);
            const float g1 = masked_diff(o && ((s.om[dc] >> fx) & 1u), s.ub[dc][fx], v);
            const float g2 = masked_diff(o && ((s.om[dz] >> fx) & 1u), s.ub[dz][fx], v);
            float out[3];
            dual_update(s.pfy[0][fw][fx], s.pfy[1][fw][fx], s.pfy[2][fw][fx], g0, g1, g2, a.sigma, out);
            s.py[r9(-1, fw)][fx] = out[1];
        }
        {  // -z face: fw is y
            const int d = r10(fw, -1), dy = r10(fw + 1, -1), dc = r10(fw, 0);
            const unsigned om = s.om[d];
            const bool o = (om >> fx) & 1u;
            const float v = s.ub[d][fx];
            const float g0 = masked_diff(o && ((om >> (fx + 1)) & 1u), fx < 7 ? s.ub[d][fx < 7 ? fx + 1 : 7] : s.xhp[d], v);
            const float g1 = masked_diff(o && ((s.om[dy] >> fx) & 1u), s.ub[dy][fx], v);
            const float g2 = masked_diff(o && ((s.om[dc] >> fx) & 1u), s.ub[dc][fx], v);
            float out[3];
            dual_update(s.pfz[0][fw][fx], s.pfz[1][fw][fx], s.pfz[2][fw][fx], g0, g1, g2, a.sigma, out);
            s.pz[r9(fw, -1)][fx] = out[2];
        }
    }
    sts_row(s.py[r9(ly, lz)], p1);
    sts_row(s.pz[r9(ly, lz)], p2);
    __syncthreads();

    // ----------------------------------------------- primal + relaxation
    {
        float pym[8], pzm[8];
        lds_row(s.py[r9(ly - 1, lz)], pym);
        lds_row(s.pz[r9(ly, lz - 1)], pzm);
        const unsigned om_ym = s.om[r10(ly - 1, lz)], om_zm = s.om[r10(ly, lz - 1)];
        const unsigned om_yp = s.om[r10(ly + 1, lz)], om_zp = s.om[r10(ly, lz + 1)];
        const float pxm = s.pxm[r];
        // edge masks of the row's voxels towards +a and from -a (bit 9 of om_r is the -x halo)
        const unsigned exp_ = om_r & (om_r >> 1), exm_ = om_r & ((om_r << 1) | ((om_r >> 9) & 1u));
        const unsigned eyp = om_r & om_yp, eym = om_r & om_ym, ezp = om_r & om_zp, ezm = om_r & om_zm;
        float un[8], ubn[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const bool o = (om_r >> x) & 1u;
            const float dv = div_terms((exp_ >> x) & 1u, p0[x], (exm_ >> x) & 1u, x > 0 ? p0[x > 0 ? x - 1 : 0] : pxm,
                                       (eyp >> x) & 1u, p1[x], (eym >> x) & 1u, pym[x],
                                       (ezp >> x) & 1u, p2[x], (ezm >> x) & 1u, pzm[x]);
            primal_update(o, uo[x], o ? dv : 0.0f, fv[x], wv[x], a.tau, a.tau_lam, a.theta, &un[x], &ubn[x]);
        }
        st_row<T>(a.u + base, un);
        st_row<T>(a.ub_out + base, ubn);
        st_row<T>(a.p_out + base, p0);
        st_row<T>(a.p_out + ps + base, p1);
        st_row<T>(a.p_out + 2 * ps + base, p2);
    }
}

// One block of the row sweep: staging of the rows, faces and edges, the dual steps,
// the primal step and the relaxation.  `stage` holds the block's own fields when they
// were prefetched into shared memory (else they are read from global memory).
template <typename T, bool ASYNC = false, bool PREFETCH = false, bool BAL = false>
__device__ __forceinline__ void rows_block(const SweepArgs<T>& a, RowTiles& s, int b, int r, const char* stage,
                                           const int* nb, HaloRaw<T>* raw = nullptr, char* slot = nullptr,
                                           int b_next = -1) {
    const int ly = r & 7, lz = r >> 3;
    const int rr = r10(ly, lz);
    const size_t ps = a.pstride;
    const size_t base = (size_t)b * kBlockVoxels + 8 * r;
    // ---------------------------------------------------------- staging
    constexpr bool kAsync = ASYNC;
    unsigned hom[4] = {0u, 0u, 0u, 0u};
    if constexpr (kAsync) issue_row_halos<T, BAL>(a, s, *raw, r, ly, lz, nb, hom);
    float ub[8], p0[8], p1[8], p2[8], uo[8], fv[8], wv[8];
    unsigned om_r;
    if constexpr (PREFETCH) {  // this block's row r is in the thread's slot (copied one block ago)
        using L = OwnSlot<T>;
        ld_row_smem<T>(reinterpret_cast<const T*>(slot + L::kUb), ub);
        ld_row_smem<T>(reinterpret_cast<const T*>(slot + L::kP), p0);
        ld_row_smem<T>(reinterpret_cast<const T*>(slot + L::kP + L::kRowT), p1);
        ld_row_smem<T>(reinterpret_cast<const T*>(slot + L::kP + 2 * L::kRowT), p2);
        ld_row_smem<T>(reinterpret_cast<const T*>(slot + L::kU), uo);
        lds_row(reinterpret_cast<const float*>(slot + L::kF), fv);
        lds_row(reinterpret_cast<const float*>(slot + L::kW), wv);
        om_r = (*reinterpret_cast<const uint32_t*>(slot + L::kBits) >> (8 * (r & 3))) & 0xffu;
        // the slot is free again: bring in the next block's row while this one computes
        if (b_next >= 0) issue_own_row<T>(a, slot, b_next, r);
        cp_async_commit();
    } else if (stage) {  // this block's rows were brought into shared memory by the bulk copies
        using L = RowStage<T>;
        ld_row_smem<T>(reinterpret_cast<const T*>(stage + L::kUb) + 8 * r, ub);
        ld_row_smem<T>(reinterpret_cast<const T*>(stage + L::kP) + 8 * r, p0);
        ld_row_smem<T>(reinterpret_cast<const T*>(stage + L::kP + L::kField) + 8 * r, p1);
        ld_row_smem<T>(reinterpret_cast<const T*>(stage + L::kP + 2 * L::kField) + 8 * r, p2);
        ld_row_smem<T>(reinterpret_cast<const T*>(stage + L::kU) + 8 * r, uo);
        lds_row(reinterpret_cast<const float*>(stage + L::kF) + 8 * r, fv);
        lds_row(reinterpret_cast<const float*>(stage + L::kW) + 8 * r, wv);
        om_r = (reinterpret_cast<const uint32_t*>(stage + L::kBits)[r >> 2] >> (8 * (r & 3))) & 0xffu;
    } else {
        ld_row<T>(a.ub_in + base, ub);
        ld_row<T>(a.p_in + base, p0);
        ld_row<T>(a.p_in + ps + base, p1);
        ld_row<T>(a.p_in + 2 * ps + base, p2);
        ld_row<T>(a.u + base, uo);
        const float4* f4 = reinterpret_cast<const float4*>(a.f + base);
        const float4* w4 = reinterpret_cast<const float4*>(a.w + base);
        const float4 fa = __ldg(f4), fb = __ldg(f4 + 1), wa = __ldg(w4), wb = __ldg(w4 + 1);
        fv[0] = fa.x, fv[1] = fa.y, fv[2] = fa.z, fv[3] = fa.w, fv[4] = fb.x, fv[5] = fb.y, fv[6] = fb.z, fv[7] = fb.w;
        wv[0] = wa.x, wv[1] = wa.y, wv[2] = wa.z, wv[3] = wa.w, wv[4] = wb.x, wv[5] = wb.y, wv[6] = wb.z, wv[7] = wb.w;
        om_r = row_bits(a.bits, b, r);
    }
    // x halos of the row: u_bar and Omega at x = 8 and x = -1, old p at x = -1
    float hm0 = 0.0f, hm1 = 0.0f, hm2 = 0.0f;
    if constexpr (kAsync) {
        om_r |= hom[0];  // the dual and primal steps read the row's bits from this register
        sts_row(s.ub[rr], ub);
        s.om[rr] = (unsigned short)om_r;
        if constexpr (!BAL) {  // (balanced items store their Omega words themselves)
            if (ly == 7) s.om[r10(8, lz)] = (unsigned short)hom[1];
            if (ly == 0) s.om[r10(-1, lz)] = (unsigned short)hom[1];
            if (lz == 7) s.om[r10(ly, 8)] = (unsigned short)hom[2];
            if (lz == 0) s.om[r10(ly, -1)] = (unsigned short)hom[2];
            if (ly == 0 && lz == 7) s.om[r10(-1, 8)] = (unsigned short)hom[3];
            if (ly == 7 && lz == 0) s.om[r10(8, -1)] = (unsigned short)hom[3];
        }
        if constexpr (PREFETCH) {
            // the halo group is complete; the next block's rows (the newest group) may
            // still be in flight
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            cp_async_wait_all();
        }
        if constexpr (sizeof(T) != 4) {
            if constexpr (BAL) convert_halos_balanced<T>(s, *raw, r, ly, lz, nb);
            else convert_row_halos<T>(s, *raw, r, ly, lz);
        }
    } else {
        {
            unsigned bit;
            const float xp = load_voxel<T>(a, nb[0], 8 * r, &bit);
            om_r |= bit << 8;
            const int n3 = nb[3];
            const float xm = load_voxel<T>(a, n3, 8 * r + 7, &bit);
            om_r |= bit << 9;
            if (n3 >= 0) {
                const size_t o3 = (size_t)n3 * kBlockVoxels + 8 * r + 7;
                hm0 = Store<T>::ld(a.p_in + o3);
                hm1 = Store<T>::ld(a.p_in + ps + o3);
                hm2 = Store<T>::ld(a.p_in + 2 * ps + o3);
            }
            s.xhp[rr] = xp;
            s.xhm[rr] = xm;
        }
        sts_row(s.ub[rr], ub);
        s.om[rr] = (unsigned short)om_r;
        // faces and edges
        if constexpr (BAL) {
            load_faces_balanced<T>(a, s, r, nb);
        } else {
            if (ly == 7) {  // row (8, lz) <- block +y row (0, lz); edge (-1, 8, lz) <- block (-x,+y) voxel (7, 0, lz)
                const int d = r10(8, lz);
                unsigned om = load_face_row<T>(a, nb[1], 8 * lz, s.ub[d]), bit;
                s.xhm[d] = load_voxel<T>(a, nb[6], 8 * (8 * lz) + 7, &bit);
                s.om[d] = (unsigned short)(om | (bit << 9));
            }
            if (ly == 0) {  // row (-1, lz) <- block -y row (7, lz); edge (8, -1, lz) <- block (-y,+x) voxel (0, 7, lz)
                const int d = r10(-1, lz);
                const int n4 = nb[4];
                unsigned om = load_face_row<T>(a, n4, 7 + 8 * lz, s.ub[d]), bit;
                s.xhp[d] = load_voxel<T>(a, nb[8], 8 * (7 + 8 * lz), &bit);
                s.om[d] = (unsigned short)(om | (bit << 8));
                float q[8];
        #pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (n4 >= 0) ld_row<T>(a.p_in + c * ps + (size_t)n4 * kBlockVoxels + 8 * (7 + 8 * lz), q);
                    else
        #pragma unroll
                        for (int i = 0; i < 8; ++i) q[i] = 0.0f;
                    sts_row(s.pfy[c][lz], q);
                }
            }
            if (lz == 7) {  // row (ly, 8) <- block +z row (ly, 0); edge (-1, ly, 8) <- block (-x,+z) voxel (7, ly, 0)
                const int d = r10(ly, 8);
                unsigned om = load_face_row<T>(a, nb[2], ly, s.ub[d]), bit;
                s.xhm[d] = load_voxel<T>(a, nb[7], 8 * ly + 7, &bit);
                s.om[d] = (unsigned short)(om | (bit << 9));
            }
            if (lz == 0) {  // row (ly, -1) <- block -z row (ly, 7); edge (8, ly, -1) <- block (-z,+x) voxel (0, ly, 7)
                const int d = r10(ly, -1);
                const int n5 = nb[5];
                unsigned om = load_face_row<T>(a, n5, ly + 56, s.ub[d]), bit;
                s.xhp[d] = load_voxel<T>(a, nb[10], 8 * (ly + 56), &bit);
                s.om[d] = (unsigned short)(om | (bit << 8));
                float q[8];
        #pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (n5 >= 0) ld_row<T>(a.p_in + c * ps + (size_t)n5 * kBlockVoxels + 8 * (ly + 56), q);
                    else
        #pragma unroll
                        for (int i = 0; i < 8; ++i) q[i] = 0.0f;
                    sts_row(s.pfz[c][ly], q);
                }
            }
            if (ly == 0 && lz == 7)  // edge row (-1, 8) <- block (-y,+z) row (7, 0)
                s.om[r10(-1, 8)] = (unsigned short)load_face_row<T>(a, nb[9], 7, s.ub[r10(-1, 8)]);
            if (ly == 7 && lz == 0)  // edge row (8, -1) <- block (-z,+y) row (0, 7)
                s.om[r10(8, -1)] = (unsigned short)load_face_row<T>(a, nb[11], 56, s.ub[r10(8, -1)]);
        }
    }
    __syncthreads();
    if constexpr (kAsync) hm0 = s.phm[0][r], hm1 = s.phm[1][r], hm2 = s.phm[2][r];
    rows_compute<T>(a, s, r, om_r, ub, p0, p1, p2, uo, fv, wv, hm0, hm1, hm2, base);
}

// Loads the neighbour row of block b (every thread reads the same 48 bytes).
__device__ inline void load_nbr_row(const int32_t* __restrict__ nbr, int b, int* out) {
    const int4* p = reinterpret_cast<const int4*>(nbr + (size_t)b * kNeighbours);
    const int4 x = __ldg(p), y = __ldg(p + 1), z = __ldg(p + 2);
    out[0] = x.x, out[1] = x.y, out[2] = x.z, out[3] = x.w, out[4] = y.x, out[5] = y.y;
    out[6] = y.z, out[7] = y.w, out[8] = z.x, out[9] = z.y, out[10] = z.z, out[11] = z.w;
}

template <typename T, int MINB, bool ASYNC = false, bool BAL = false>
__global__ void __launch_bounds__(kRowThreads, MINB) sweep_rows_kernel(SweepArgs<T> a) {
    __shared__ RowTiles s;
    __shared__ HaloRaw<T> raw;
    const int G = gridDim.x;
    int k = blockIdx.x;
    if (k >= a.n_blocks) return;
    // the next block's index and neighbour row are fetched one block ahead, so that a
    // block's halo loads do not wait behind two dependent round trips
    int b = a.order ? __ldg(a.order + k) : k;
    int nb[kNeighbours], nb_next[kNeighbours];
    load_nbr_row(a.nbr, b, nb);
    for (; k < a.n_blocks; k += G) {
        const int kn = k + G;
        int b_next = -1;
        if (kn < a.n_blocks) {
            b_next = a.order ? __ldg(a.order + kn) : kn;
            load_nbr_row(a.nbr, b_next, nb_next);
        }
        rows_block<T, ASYNC, false, BAL>(a, s, b, threadIdx.x, nullptr, nb, &raw);
        __syncthreads();  // the tiles are rewritten for the next block
        b = b_next;
#pragma unroll
        for (int i = 0; i < kNeighbours; ++i) nb[i] = nb_next[i];
    }
}

// Row sweep with asynchronous halos and the next block's own rows prefetched: while a
// CTA computes block k, every thread's copies of its row of block k + grid are already
// in flight into its stage slot, so the DRAM latency of a block's own fields overlaps
// the previous block's arithmetic instead of following it.  Same arithmetic as every
// other variant (bit-identical iterates).
template <typename T, int MINB>
__global__ void __launch_bounds__(kRowThreads, MINB) sweep_rows_prefetch_kernel(SweepArgs<T> a) {
    __shared__ RowTiles s;
    __shared__ HaloRaw<T> raw;
    __shared__ __align__(16) char stage[kRowThreads * OwnSlot<T>::kBytes];
    const int G = gridDim.x;
    const int r = threadIdx.x;
    char* slot = stage + r * OwnSlot<T>::kBytes;
    int k = blockIdx.x;
    if (k >= a.n_blocks) return;
    int b = a.order ? __ldg(a.order + k) : k;
    int nb[kNeighbours], nb_next[kNeighbours];
    load_nbr_row(a.nbr, b, nb);
    issue_own_row<T>(a, slot, b, r);
    cp_async_commit();
    for (; k < a.n_blocks; k += G) {
        const int kn = k + G;
        int b_next = -1;
        if (kn < a.n_blocks) {
            b_next = a.order ? __ldg(a.order + kn) : kn;
            load_nbr_row(a.nbr, b_next, nb_next);
        }
        cp_async_wait_all();  // this block's own rows (and nothing else) were pending
        rows_block<T, true, true>(a, s, b, r, nullptr, nb, &raw, slot, b_next);
        __syncthreads();  // the tiles are rewritten for the next block
        b = b_next;
#pragma unroll
        for (int i = 0; i < kNeighbours; ++i) nb[i] = nb_next[i];
    }
}

// One thread's row of a block's own fields as stored (16-byte words), loaded ahead of use.
template <typename T>
struct OwnRows {
    static constexpr int R = sizeof(T) == 4 ? 2 : 1;  // 16-byte words per row of 8 values
    uint4 ub[R], p[3][R], u[R];
    float4 f[2], w[2];
    unsigned bits;  // the row's Omega byte
};

template <typename T>
__device__ __forceinline__ void load_own_rows(const SweepArgs<T>& a, int b, int r, OwnRows<T>& o) {
    constexpr int R = OwnRows<T>::R;
    const size_t base = (size_t)b * kBlockVoxels + 8 * r;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        o.ub[i] = __ldg(reinterpret_cast<const uint4*>(a.ub_in + base) + i);
#pragma unroll
        for (int c = 0; c < 3; ++c) o.p[c][i] = __ldg(reinterpret_cast<const uint4*>(a.p_in + c * a.pstride + base) + i);
        o.u[i] = __ldg(reinterpret_cast<const uint4*>(a.u + base) + i);
    }
    o.f[0] = __ldg(reinterpret_cast<const float4*>(a.f + base));
    o.f[1] = __ldg(reinterpret_cast<const float4*>(a.f + base) + 1);
    o.w[0] = __ldg(reinterpret_cast<const float4*>(a.w + base));
    o.w[1] = __ldg(reinterpret_cast<const float4*>(a.w + base) + 1);
    o.bits = row_bits(a.bits, b, r);
}

template <typename T>
__device__ __forceinline__ void unpack_row(const uint4* q, float* v) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            v[4 * i] = __uint_as_float(q[i].x), v[4 * i + 1] = __uint_as_float(q[i].y);
            v[4 * i + 2] = __uint_as_float(q[i].z), v[4 * i + 3] = __uint_as_float(q[i].w);
        }
    } else {
        unpack8<T>(q[0], v);
    }
}

__device__ __forceinline__ void unpack_f4(const float4* q, float* v) {
    v[0] = q[0].x, v[1] = q[0].y, v[2] = q[0].z, v[3] = q[0].w;
    v[4] = q[1].x, v[5] = q[1].y, v[6] = q[1].z, v[7] = q[1].w;
}

// Software-pipelined row sweep: while a CTA computes block k from one tile set, the
// halos of block k + grid are already being copied (cp.async) into the other tile set,
// and every thread's own row of that block is in flight into registers.  A block's
// data is therefore requested one whole block ahead, and a CTA's critical path is its
// arithmetic rather than its memory round trips.  Same arithmetic as every other
// variant (bit-identical iterates).
template <typename T, int MINB, bool BAL = false>
__global__ void __launch_bounds__(kRowThreads, MINB) sweep_rows_pipelined_kernel(SweepArgs<T> a) {
    __shared__ RowTiles tiles[2];
    __shared__ HaloRaw<T> raws[2];
    const int G = gridDim.x;
    const int r = threadIdx.x, ly = r & 7, lz = r >> 3, rr = r10(ly, lz);
    int k = blockIdx.x;
    if (k >= a.n_blocks) return;
    int b = a.order ? __ldg(a.order + k) : k;
    int nb[kNeighbours], nb_next[kNeighbours];
    load_nbr_row(a.nbr, b, nb);
    OwnRows<T> own, own_next;
    unsigned hom[4], hom_next[4];
    issue_row_halos<T, BAL>(a, tiles[0], raws[0], r, ly, lz, nb, hom);
    load_own_rows<T>(a, b, r, own);
    for (int i = 0; k < a.n_blocks; k += G, ++i) {
        RowTiles& S = tiles[i & 1];
        const int kn = k + G;
        int b_next = -1;
        if (kn < a.n_blocks) {
            b_next = a.order ? __ldg(a.order + kn) : kn;
            load_nbr_row(a.nbr, b_next, nb_next);
        }
        float ub[8], p0[8], p1[8], p2[8], uo[8], fv[8], wv[8];
        unpack_row<T>(own.ub, ub);
        unpack_row<T>(own.p[0], p0);
        unpack_row<T>(own.p[1], p1);
        unpack_row<T>(own.p[2], p2);
        unpack_row<T>(own.u, uo);
        unpack_f4(own.f, fv);
        unpack_f4(own.w, wv);
        const unsigned om_r = own.bits | hom[0];
        // the next block goes in flight: its halos into the other tile set (free since the
        // barrier that ended the previous block), its own row into registers
        if (b_next >= 0) {
            issue_row_halos<T, BAL>(a, tiles[(i & 1) ^ 1], raws[(i & 1) ^ 1], r, ly, lz, nb_next, hom_next);
            load_own_rows<T>(a, b_next, r, own_next);
        } else {
            cp_async_commit();  // an empty group: the wait below then always leaves the newest group
        }
        sts_row(S.ub[rr], ub);
        S.om[rr] = (unsigned short)om_r;
        if constexpr (!BAL) {  // (balanced items stored their Omega words when issued)
            if (ly == 7) S.om[r10(8, lz)] = (unsigned short)hom[1];
            if (ly == 0) S.om[r10(-1, lz)] = (unsigned short)hom[1];
            if (lz == 7) S.om[r10(ly, 8)] = (unsigned short)hom[2];
            if (lz == 0) S.om[r10(ly, -1)] = (unsigned short)hom[2];
            if (ly == 0 && lz == 7) S.om[r10(-1, 8)] = (unsigned short)hom[3];
            if (ly == 7 && lz == 0) S.om[r10(8, -1)] = (unsigned short)hom[3];
        }
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this block's halos have landed
        if constexpr (sizeof(T) != 4) {
            if constexpr (BAL) convert_halos_balanced<T>(S, raws[i & 1], r, ly, lz, nb);
            else convert_row_halos<T>(S, raws[i & 1], r, ly, lz);
        }
        __syncthreads();
        const float hm0 = S.phm[0][r], hm1 = S.phm[1][r], hm2 = S.phm[2][r];
        rows_compute<T>(a, S, r, om_r, ub, p0, p1, p2, uo, fv, wv, hm0, hm1, hm2, (size_t)b * kBlockVoxels + 8 * r);
        __syncthreads();  // this tile set is refilled for the block after next
        b = b_next;
#pragma unroll
        for (int q = 0; q < kNeighbours; ++q) nb[q] = nb_next[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) hom[q] = hom_next[q];
        own = own_next;
    }
}

// ------------------------------------------------------- row sweep with TMA
// The row sweep with the next block's own fields prefetched: while a CTA computes
// block k, one thread has already issued 1-D bulk copies (cp.async.bulk, the TMA
// engine) of block k + grid into the other half of a double-buffered stage, completing
// on that half's mbarrier.  The waits are bounded: a copy that never lands sets the
// timeout flag and the CTA stops instead of spinning forever.
__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((unsigned)__cvta_generic_to_shared(bar)), "r"(count)
                 : "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"((unsigned)__cvta_generic_to_shared(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ inline void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes), "r"((unsigned)__cvta_generic_to_shared(bar))
                 : "memory");
}

template <typename T>
__device__ inline void stage_issue(const SweepArgs<T>& a, char* dst, int b, uint64_t* bar) {
    using L = RowStage<T>;
    const size_t v0 = (size_t)b * kBlockVoxels;
    // order earlier generic reads of this half before the asynchronous writes into it
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, L::kTx);
    bulk_load(dst + L::kUb, a.ub_in + v0, L::kField, bar);
#pragma unroll
    for (int c = 0; c < 3; ++c) bulk_load(dst + L::kP + c * L::kField, a.p_in + c * a.pstride + v0, L::kField, bar);
    bulk_load(dst + L::kU, a.u + v0, L::kField, bar);
    bulk_load(dst + L::kF, a.f + v0, kBlockVoxels * 4, bar);
    bulk_load(dst + L::kW, a.w + v0, kBlockVoxels * 4, bar);
    bulk_load(dst + L::kBits, a.bits + (size_t)b * 16, 64, bar);
}

constexpr long long kWaitLimit = 1ll << 22;  // try_wait rounds before a wait counts as lost

template <typename T>
__global__ void __launch_bounds__(kRowThreads, 4) sweep_rows_tma_kernel(SweepArgs<T> a) {
    using L = RowStage<T>;
    __shared__ RowTiles s;
    __shared__ HaloRaw<T> raw;
    __shared__ __align__(8) uint64_t bars[2];
    extern __shared__ __align__(128) char stages[];  // [2][L::kBytes]
    const int t = threadIdx.x;
    const int G = gridDim.x;
    int k = blockIdx.x;
    if (k >= a.n_blocks) return;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    auto block_at = [&](int kk) { return a.order ? __ldg(a.order + kk) : kk; };
    if (t == 0) stage_issue<T>(a, stages, block_at(k), &bars[0]);
    unsigned parity[2] = {0u, 0u};
    for (int i = 0; k < a.n_blocks; ++i, k += G) {
        const int h = i & 1;
        if (t == 0 && k + G < a.n_blocks) stage_issue<T>(a, stages + (h ^ 1) * L::kBytes, block_at(k + G), &bars[h ^ 1]);
        long long it = 0;
        while (!mbar_try_wait(&bars[h], parity[h]) && ++it < kWaitLimit) {
        }
        if (it >= kWaitLimit) {
            if (t == 0) atomicOr(a.err, kErrTimeout);
            return;
        }
        parity[h] ^= 1u;
        const int b = block_at(k);
        int nb[kNeighbours];
        load_nbr_row(a.nbr, b, nb);
        rows_block<T, true>(a, s, b, t, stages + h * L::kBytes, nb, &raw);
        __syncthreads();  // tiles and this stage half are reused
    }
}

template <typename T>
constexpr size_t sweep_pipe_smem() {
    return ((sizeof(Tiles) + 15) / 16) * 16 + 2 * StageLayout<T>::kBytes + 3 * kNeighbours * sizeof(int);
}

// sqrt(x) for the primal energy: the single-precision reciprocal square root (rsqrtf,
// within 2 ulps) gives s0 = x r, one step of Heron's method (Newton's iteration for
// s^2 = x), s1 = s0 + (x - s0^2) r / 2 in float64, squares its relative error (about
// 2^-44 left, below the parity tolerance of the energies); x too small for single
// precision takes the float64 square root.
__device__ __forceinline__ double energy_sqrt(double x) {
    if (!(x > 1.0e-30)) return sqrt(x);
    const float r = rsqrtf((float)x);
    const double s0 = (double)((float)x * r);
    return fma(0.5 * (double)r, fma(-s0, s0, x), s0);
}

template <typename T>
__global__ void __launch_bounds__(kSweepThreads) energy_kernel(const T* __restrict__ u, const T* __restrict__ p,
                                                               const float* __restrict__ f,
                                                               const float* __restrict__ w,
                                                               const uint32_t* __restrict__ bits,
                                                               const int32_t* __restrict__ nbr, size_t pstride,
                                                               int n_blocks, double lam,
                                                               const double* __restrict__ inv2lw, double* partials) {
    __shared__ Tiles s;
    __shared__ double red[2][kSweepThreads / 32];
    const int t = threadIdx.x;
    const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
    double accP = 0.0, accD = 0.0;
    for (int b = blockIdx.x; b < n_blocks; b += gridDim.x) {
        float uc;
        bool oc;
        stage_tiles<T>(s, b, u, p, pstride, bits, nbr, t, lx, ly, lz, uc, oc);
        if (oc) {
            const int c = t10(lx, ly, lz);
            const double u0 = uc;
            double tv2 = 0.0;
            const int step[3] = {1, kTile, kTile * kTile};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (s.om[c + step[a]]) {
                    const double g = (double)s.v[c + step[a]] - u0;
                    tv2 += g * g;
                }
            }
            const size_t v = (size_t)b * kBlockVoxels + t;
            const float wf = w[v];
            const double fv = f[v], wv = wf;
            const double r = u0 - fv;
            accP += energy_sqrt(tv2) + 0.5 * lam * wv * r * r;
            const int q = t9(lx, ly, lz);
            const int pstep[3] = {1, kPTile, kPTile * kPTile};
            double dv = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double own = s.om[c + step[a]] ? (double)s.p[a][q] : 0.0;
                const double back = s.om[c - step[a]] ? (double)s.p[a][q - pstep[a]] : 0.0;
                dv += own - back;
            }
            // 1/(2 lambda w) from the table for integer counts (the fusion's weights), else divided
            const int wi = (int)wf;
            const double inv = ((float)wi == wf && wi >= 1 && wi <= kInvWeights) ? __ldg(inv2lw + wi - 1)
                                                                                 : 1.0 / (2.0 * lam * wv);
            accD += -fv * dv - dv * dv * inv;
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) {
        accP += __shfl_xor_sync(0xffffffffu, accP, o);
        accD += __shfl_xor_sync(0xffffffffu, accD, o);
    }
    if ((t & 31) == 0) red[0][t >> 5] = accP, red[1][t >> 5] = accD;
    __syncthreads();
    if (t == 0) {
        double P = 0.0, D = 0.0;
        for (int i = 0; i < kSweepThreads / 32; ++i) P += red[0][i], D += red[1][i];
        partials[2 * blockIdx.x] = P;
        partials[2 * blockIdx.x + 1] = D;
    }
}

__global__ void __launch_bounds__(1024) energy_final_kernel(double* partials, int n) {
    __shared__ double rp[1024], rd[1024];
    double P = 0.0, D = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) P += partials[2 * i], D += partials[2 * i + 1];
    rp[threadIdx.x] = P, rd[threadIdx.x] = D;
    __syncthreads();
    for (int sft = blockDim.x / 2; sft > 0; sft >>= 1) {
        if ((int)threadIdx.x < sft) rp[threadIdx.x] += rp[threadIdx.x + sft], rd[threadIdx.x] += rd[threadIdx.x + sft];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[2 * n] = rp[0], partials[2 * n + 1] = rd[0];
}

__global__ void omega_bits_kernel(const float* __restrict__ w, uint32_t* bits, int n_blocks) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int b = warp; b < n_blocks; b += nwarps) {
        for (int k = 0; k < 16; ++k) {
            const bool o = __ldg(w + (size_t)b * kBlockVoxels + 32 * k + lane) > 0.0f;
            const unsigned word = __ballot_sync(0xffffffffu, o);
            if (lane == 0) bits[(size_t)b * 16 + k] = word;
        }
    }
}

__global__ void neighbours_kernel(DeviceMap m, int n_blocks) {
    const long long total = (long long)n_blocks * kNeighbours;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / kNeighbours), e = (int)(i % kNeighbours);
        const int4 k = reinterpret_cast<const int4*>(m.coords)[b];
        int dx, dy, dz;
        neighbour_offset(e, &dx, &dy, &dz);
        int32_t idx = -1;
        if (key_in_range(k.x, (long long)k.y + dx, (long long)k.z + dy, (long long)k.w + dz)) {
            idx = hash_lookup(m, pack_key(k.x, k.y + dx, k.z + dy, k.w + dz));
            if (idx >= n_blocks) idx = -1;
        }
        m.nbr[i] = idx;
    }
}

__global__ void omega_bytes_kernel(const float* __restrict__ w, uint8_t* out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = w[i] > 0.0f ? 1 : 0;
}

template <typename T>
__global__ void convert_kernel(const void* src, void* dst, long long n, int to_float) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (to_float) reinterpret_cast<float*>(dst)[i] = Store<T>::ld(reinterpret_cast<const T*>(src) + i);
        else Store<T>::st(reinterpret_cast<T*>(dst) + i, reinterpret_cast<const float*>(src)[i]);
    }
}

// Launches a row sweep with registers for MINB resident CTAs per SM, as many CTAs as are
// resident at once (at most one per block).
template <typename T, int MINB, bool ASYNC, bool BAL>
void launch_rows(const SweepArgs<T>& a, int64_t nb, int sm_count, cudaStream_t s) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_kernel<T, MINB, ASYNC, BAL>, kRowThreads, 0);
    const int grid = (int)std::min<int64_t>(nb, (int64_t)sm_count * std::max(per_sm, 1));
    sweep_rows_kernel<T, MINB, ASYNC, BAL><<<grid, kRowThreads, 0, s>>>(a);
}

template <typename T>
void sweep_t(denser_ctx* c, int64_t nb, cudaStream_t s) {
    SweepArgs<T> a;
    const int cur = c->cur;
    a.ub_in = (const T*)c->d.ub[cur];
    a.ub_out = (T*)c->d.ub[cur ^ 1];
    a.u = (T*)c->d.u;
    a.p_in = (const T*)c->d.p[cur];
    a.p_out = (T*)c->d.p[cur ^ 1];
    a.f = c->d.f;
    a.w = c->d.w;
    a.bits = c->d.omega_bits;
    a.nbr = c->d.nbr;
    a.pstride = (size_t)c->d.max_blocks * kBlockVoxels;
    a.n_blocks = (int)nb;
    a.sigma = (float)c->prm.sigma;
    a.tau = (float)c->prm.tau;
    a.tau_lam = (float)(c->prm.tau * c->prm.lambda);
    a.theta = (float)c->prm.theta;
    a.order = c->sched.order ? c->order : nullptr;
    a.err = c->d.counters + kErrorBits;
    if (c->sched.sweep_kernel == 0) {
        const int per_sm = c->sched.ctas_per_sm > 0 ? c->sched.ctas_per_sm : 4;
        const int grid = (int)std::min<int64_t>(nb, (int64_t)c->sm_count * per_sm);
        sweep_kernel<T><<<grid, kSweepThreads, 0, s>>>(a);
    } else if (c->sched.sweep_kernel == 2) {
        // ctas_per_sm selects the register budget: 0 / 1: up to 8 resident CTAs per SM
        // (128 registers), 2: 10 (96 registers), 3: 12
        int per_sm = 0;
        switch (c->sched.ctas_per_sm) {
            case 2:
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_kernel<T, 10>, kRowThreads, 0);
                sweep_rows_kernel<T, 10><<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)),
                                           kRowThreads, 0, s>>>(a);
                break;
            case 3:
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_kernel<T, 12>, kRowThreads, 0);
                sweep_rows_kernel<T, 12><<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)),
                                           kRowThreads, 0, s>>>(a);
                break;
            default:
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_kernel<T, 8>, kRowThreads, 0);
                sweep_rows_kernel<T, 8><<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)),
                                          kRowThreads, 0, s>>>(a);
        }
    } else if (c->sched.sweep_kernel == 4) {
        // row sweep with the halos staged asynchronously
        // (ctas_per_sm 2: up to 10 resident CTAs per SM, 96 registers; 3: 12, 80 registers)
        int per_sm = 0;
        if (c->sched.ctas_per_sm == 3) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_kernel<T, 12, true>, kRowThreads, 0);
            sweep_rows_kernel<T, 12, true><<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)),
                                             kRowThreads, 0, s>>>(a);
        } else if (c->sched.ctas_per_sm == 2) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_kernel<T, 10, true>, kRowThreads, 0);
            sweep_rows_kernel<T, 10, true><<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)),
                                             kRowThreads, 0, s>>>(a);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_kernel<T, 8, true>, kRowThreads, 0);
            sweep_rows_kernel<T, 8, true><<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)),
                                            kRowThreads, 0, s>>>(a);
        }
    } else if (c->sched.sweep_kernel == 6) {
        // software-pipelined row sweep: ctas_per_sm 1 -> registers for 5 resident CTAs,
        // 3 -> 7, otherwise 6
        int per_sm = 0;
        if (c->sched.ctas_per_sm == 1) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_pipelined_kernel<T, 5>, kRowThreads, 0);
            sweep_rows_pipelined_kernel<T, 5>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        } else if (c->sched.ctas_per_sm == 3) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_pipelined_kernel<T, 7>, kRowThreads, 0);
            sweep_rows_pipelined_kernel<T, 7>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_pipelined_kernel<T, 6>, kRowThreads, 0);
            sweep_rows_pipelined_kernel<T, 6>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        }
    } else if (c->sched.sweep_kernel == 5) {
        // prefetching row sweep (about 27 KB of shared memory per CTA): ctas_per_sm 2 caps
        // the registers for 10 resident CTAs, otherwise for 8
        int per_sm = 0;
        if (c->sched.ctas_per_sm == 2) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_prefetch_kernel<T, 10>, kRowThreads, 0);
            sweep_rows_prefetch_kernel<T, 10>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_prefetch_kernel<T, 8>, kRowThreads, 0);
            sweep_rows_prefetch_kernel<T, 8>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        }
    } else if (c->sched.sweep_kernel == 9) {
        // the software-pipelined row sweep with balanced face items (ctas_per_sm as for 6)
        int per_sm = 0;
        if (c->sched.ctas_per_sm == 1) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_pipelined_kernel<T, 5, true>, kRowThreads, 0);
            sweep_rows_pipelined_kernel<T, 5, true>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        } else if (c->sched.ctas_per_sm == 3) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_pipelined_kernel<T, 7, true>, kRowThreads, 0);
            sweep_rows_pipelined_kernel<T, 7, true>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_pipelined_kernel<T, 6, true>, kRowThreads, 0);
            sweep_rows_pipelined_kernel<T, 6, true>
                <<<(int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1)), kRowThreads, 0, s>>>(a);
        }
    } else if (c->sched.sweep_kernel == 7 || c->sched.sweep_kernel == 8) {
        // row sweep with the face halos staged as balanced items: 7 asynchronously, 8
        // through registers (ctas_per_sm 2: registers for 10 resident CTAs, 3: 12, else 8)
        const int cps = c->sched.ctas_per_sm;
        if (c->sched.sweep_kernel == 7) {
            if (cps == 3) launch_rows<T, 12, true, true>(a, nb, c->sm_count, s);
            else if (cps == 2) launch_rows<T, 10, true, true>(a, nb, c->sm_count, s);
            else launch_rows<T, 8, true, true>(a, nb, c->sm_count, s);
        } else {
            if (cps == 3) launch_rows<T, 12, false, true>(a, nb, c->sm_count, s);
            else if (cps == 2) launch_rows<T, 10, false, true>(a, nb, c->sm_count, s);
            else launch_rows<T, 8, false, true>(a, nb, c->sm_count, s);
        }
    } else if (c->sched.sweep_kernel == 3) {
        int per_sm = 0;
        const size_t smem = 2 * (size_t)RowStage<T>::kBytes;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_rows_tma_kernel<T>, kRowThreads, smem);
        if (c->sched.ctas_per_sm > 0) per_sm = std::min(per_sm, 2 * c->sched.ctas_per_sm);
        const int grid = (int)std::min<int64_t>(nb, (int64_t)c->sm_count * std::max(per_sm, 1));
        sweep_rows_tma_kernel<T><<<grid, kRowThreads, smem, s>>>(a);
    } else {
        const int per_sm = c->sched.ctas_per_sm > 0 ? c->sched.ctas_per_sm : 2;
        const int grid = (int)std::min<int64_t>(nb, (int64_t)c->sm_count * per_sm);
        sweep_pipe_kernel<T><<<grid, kSweepThreads, sweep_pipe_smem<T>(), s>>>(a);
    }
}

template <typename T>
void energy_t(denser_ctx* c, int64_t nb, cudaStream_t s) {
    const int cur = c->cur;
    energy_kernel<T><<<kEnergyGrid, kSweepThreads, 0, s>>>(
        (const T*)c->d.u, (const T*)c->d.p[cur], c->d.f, c->d.w, c->d.omega_bits, c->d.nbr,
        (size_t)c->d.max_blocks * kBlockVoxels, (int)nb, c->prm.lambda, c->d.partials + 2 * kEnergyGrid + 2,
        c->d.partials);
    energy_final_kernel<<<1, 1024, 0, s>>>(c->d.partials, kEnergyGrid);
}

}  // namespace

// Tail of one body pass of the graph-captured loop: counts the k iterations just run,
// records the energies when they were evaluated, and sets the WHILE condition: run the
// body again while k more iterations fit and the relative gap is above the tolerance.
__global__ void loop_decide_kernel(const double* energy, int32_t* ci, double* cd, cudaGraphConditionalHandle h, int k,
                                   int with_gap) {
    const int done = ci[0] + k;
    ci[0] = done;
    bool more = done + k <= ci[1];
    if (with_gap) {
        const double P = energy[0], D = energy[1];
        cd[1] = P, cd[2] = D;
        ci[3] += 1;
        const bool conv = (P - D) <= cd[0] * fabs(P);
        ci[2] = conv;
        more = more && !conv;
    }
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

void release_graph_loop(denser_ctx* c) {
    if (c->loop.valid) {
        cudaGraphExecDestroy(c->loop.exec);
        cudaGraphDestroy(c->loop.graph);
    }
    c->loop.valid = false;
}

// Runs k-iteration body passes (k even, so the ping-pong buffers end where they began)
// inside one WHILE conditional node until fewer than k iterations remain or the gap
// test passes.  ctl_i / ctl_d must hold {0, max, 0, 0} / {tol, ...} on the stream.
int launch_graph_loop(denser_ctx* c, int64_t nb, int k, bool with_gap, cudaStream_t s) {
    const bool same = c->loop.valid && c->loop.nb == nb && c->loop.cur == c->cur && c->loop.k == k &&
                      c->loop.with_gap == (int)with_gap && memcmp(&c->loop.sched, &c->sched, sizeof(c->sched)) == 0;
    if (!same) {
        release_graph_loop(c);
        cudaGraph_t g;
        int rc = cuda_check(c, cudaGraphCreate(&g, 0), "cudaGraphCreate");
        if (rc) return rc;
        cudaGraphConditionalHandle h;
        rc = cuda_check(c, cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault), "conditional handle");
        // the parameter union has no usable default constructor: zeroed raw storage
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        memset(raw, 0, sizeof(raw));
        cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
        np->type = cudaGraphNodeTypeConditional;
        np->conditional.handle = h;
        np->conditional.type = cudaGraphCondTypeWhile;
        np->conditional.size = 1;
        cudaGraphNode_t node;
        if (!rc) rc = cuda_check(c, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, np), "conditional node");
        if (rc) {
            cudaGraphDestroy(g);
            return rc;
        }
        cudaGraph_t body = np->conditional.phGraph_out[0];
        cudaStream_t cs = c->capture_stream;
        rc = cuda_check(c, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                        "begin capture");
        const unsigned long long launches0 = c->launches;
        for (int i = 0; i < k && !rc; ++i) rc = launch_sweep(c, nb, cs);
        if (!rc && with_gap) rc = launch_energy(c, nb, cs);
        if (!rc) {
            loop_decide_kernel<<<1, 1, 0, cs>>>(c->d.partials + 2 * kEnergyGrid, c->ctl_i, c->ctl_d, h, k, (int)with_gap);
            rc = cuda_check(c, cudaGetLastError(), "decide kernel");
        }
        cudaGraph_t captured;
        const cudaError_t e = cudaStreamEndCapture(cs, &captured);
        c->launches = launches0;  // recording launches nothing
        if (!rc) rc = cuda_check(c, e, "end capture");
        cudaGraphExec_t exec;
        if (!rc) rc = cuda_check(c, cudaGraphInstantiate(&exec, g, 0), "graph instantiate");
        if (rc) {
            cudaGraphDestroy(g);
            return rc;
        }
        c->loop.valid = true;
        c->loop.nb = nb;
        c->loop.sched = c->sched;
        c->loop.cur = c->cur;
        c->loop.k = k;
        c->loop.with_gap = (int)with_gap;
        c->loop.graph = g;
        c->loop.exec = exec;
    }
    // the launch counter counts kernels run: known only after the loop ends (see caller)
    return cuda_check(c, cudaGraphLaunch(c->loop.exec, s), "graph launch");
}

int configure_kernels(denser_ctx* c) {
    cudaError_t e = cudaFuncSetAttribute(sweep_pipe_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep_pipe_smem<float>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_pipe_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sweep_pipe_smem<__half>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_pipe_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sweep_pipe_smem<__nv_bfloat16>());
    return cuda_check(c, e, "configure sweep kernels");
}

int launch_prepare_regularize(denser_ctx* c, int64_t nb, bool rebuild_nbr, cudaStream_t s) {
    if (nb <= 0) return DENSER_OK;
    if (c->sched.order && c->order_valid_blocks != nb) {
        int rc = launch_block_order(c, nb, s);
        if (rc) return rc;
    }
    omega_bits_kernel<<<grid_for(c->sm_count, nb * 32, 256, 8), 256, 0, s>>>(c->d.w, c->d.omega_bits, (int)nb);
    c->launches += 1;
    if (rebuild_nbr) {
        neighbours_kernel<<<grid_for(c->sm_count, nb * kNeighbours, 256, 8), 256, 0, s>>>(c->d, (int)nb);
        c->launches += 1;
        c->nbr_valid_blocks = nb;
    }
    return cuda_check(c, cudaGetLastError(), "omega / neighbour kernels");
}

int launch_sweep(denser_ctx* c, int64_t nb, cudaStream_t s) {
    if (nb <= 0) return DENSER_OK;
    switch (c->prm.precision) {
        case DENSER_FP16: sweep_t<__half>(c, nb, s); break;
        case DENSER_BF16: sweep_t<__nv_bfloat16>(c, nb, s); break;
        default: sweep_t<float>(c, nb, s); break;
    }
    c->cur ^= 1;
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "sweep kernel");
}

int launch_energy(denser_ctx* c, int64_t nb, cudaStream_t s) {
    switch (c->prm.precision) {
        case DENSER_FP16: energy_t<__half>(c, nb, s); break;
        case DENSER_BF16: energy_t<__nv_bfloat16>(c, nb, s); break;
        default: energy_t<float>(c, nb, s); break;
    }
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "energy kernels");
}

int launch_omega_bytes(denser_ctx* c, int64_t nb, uint8_t* out, cudaStream_t s) {
    const long long n = nb * kBlockVoxels;
    omega_bytes_kernel<<<grid_for(c->sm_count, n, 256, 8), 256, 0, s>>>(c->d.w, out, n);
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "omega bytes kernel");
}

int launch_convert_state(denser_ctx* c, const void* src, float* dst, int64_t n, bool to_float, cudaStream_t s) {
    const int g = grid_for(c->sm_count, n, 256, 8);
    switch (c->prm.precision) {
        case DENSER_FP16: convert_kernel<__half><<<g, 256, 0, s>>>(src, dst, n, to_float); break;
        case DENSER_BF16: convert_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(src, dst, n, to_float); break;
        default: convert_kernel<float><<<g, 256, 0, s>>>(src, dst, n, to_float); break;
    }
    c->launches += 1;
    return cuda_check(c, cudaGetLastError(), "convert kernel");
}

}  // namespace denser
