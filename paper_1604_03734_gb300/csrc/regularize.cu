// Omega-aware primal-dual regularisation (Section III-B, Eq. 3 and Eq. 4; Section III-C).
//
// Per regularisation call:
//   omega_bits   Omega = {w > 0} packed 32 voxels per word (ballot per warp);
//   neighbours   per block the indices of its 6 face and 6 (low, high) edge
//                neighbours through the hash table (-1: unallocated = Omega-bar);
// per iteration, one fused sweep:
//   sweep        one CTA per 8^3 block (grid-stride), one thread per voxel.  The CTA
//                stages u_bar on the block, its six faces and six edges, Omega on the
//                same positions and p on the block and its three low faces in shared
//                memory (the "block as a grid whose boundary conditions come from its
//                neighbours' I_Omega", Section III-B).  It then takes the dual step on the
//                block and on its low faces (the divergence needs p^{k+1} one voxel
//                behind), synchronises, and takes the primal step and the relaxation.
//                u_bar and p are ping-ponged across iterations; u is updated in place.
// and on demand:
//   energy       FP64 primal P(u) and dual D(p) partial sums per CTA (fixed grid, fixed
//                order: deterministic), then one CTA sums the partials.
#include <math.h>

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

// Dual step at tile position (x, y, z): p <- P(p + sigma grad_Omega u_bar), Eq. 3.
__device__ inline void dual_step(Tiles& s, int x, int y, int z, float sigma, float* out) {
    const int c = t10(x, y, z);
    const bool o = s.om[c];
    const float u0 = s.v[c];
    const float g0 = (o && s.om[c + 1]) ? s.v[c + 1] - u0 : 0.0f;
    const float g1 = (o && s.om[c + kTile]) ? s.v[c + kTile] - u0 : 0.0f;
    const float g2 = (o && s.om[c + kTile * kTile]) ? s.v[c + kTile * kTile] - u0 : 0.0f;
    const int q = t9(x, y, z);
    const float q0 = s.p[0][q] + sigma * g0;
    const float q1 = s.p[1][q] + sigma * g1;
    const float q2 = s.p[2][q] + sigma * g2;
    const float m = fmaxf(1.0f, sqrtf(q0 * q0 + q1 * q1 + q2 * q2));
    out[0] = q0 / m, out[1] = q1 / m, out[2] = q2 / m;
}

// Omega-aware divergence at a block voxel, Eq. 4 as the negative adjoint of Eq. 3.
__device__ inline float divergence(const Tiles& s, int x, int y, int z) {
    const int c = t10(x, y, z);
    const int q = t9(x, y, z);
    const bool o = s.om[c];
    const float d0 = ((o && s.om[c + 1]) ? s.p[0][q] : 0.0f) - ((o && s.om[c - 1]) ? s.p[0][q - 1] : 0.0f);
    const float d1 = ((o && s.om[c + kTile]) ? s.p[1][q] : 0.0f) -
                     ((o && s.om[c - kTile]) ? s.p[1][q - kPTile] : 0.0f);
    const float d2 = ((o && s.om[c + kTile * kTile]) ? s.p[2][q] : 0.0f) -
                     ((o && s.om[c - kTile * kTile]) ? s.p[2][q - kPTile * kPTile] : 0.0f);
    return (d0 + d1) + d2;
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
        float un = uo;
        if (oc) {
            const float ut = uo + a.tau * divergence(s, lx, ly, lz);
            const float tlw = a.tau_lam * wv;
            un = (ut + tlw * fv) / (1.0f + tlw);
        }
        const float ubn = un + a.theta * (un - uo);
        Store<T>::st(a.u + v, un);
        Store<T>::st(a.ub_out + v, ubn);
#pragma unroll
        for (int c = 0; c < 3; ++c) Store<T>::st(a.p_out + c * a.pstride + v, pc[c]);
        __syncthreads();  // the tiles are reused by the next block
    }
}

template <typename T>
__global__ void __launch_bounds__(kSweepThreads) energy_kernel(const T* __restrict__ u, const T* __restrict__ p,
                                                               const float* __restrict__ f,
                                                               const float* __restrict__ w,
                                                               const uint32_t* __restrict__ bits,
                                                               const int32_t* __restrict__ nbr, size_t pstride,
                                                               int n_blocks, double lam, double* partials) {
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
            const double fv = f[v], wv = w[v];
            const double r = u0 - fv;
            accP += sqrt(tv2) + 0.5 * lam * wv * r * r;
            const int q = t9(lx, ly, lz);
            const int pstep[3] = {1, kPTile, kPTile * kPTile};
            double dv = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double own = s.om[c + step[a]] ? (double)s.p[a][q] : 0.0;
                const double back = s.om[c - step[a]] ? (double)s.p[a][q - pstep[a]] : 0.0;
                dv += own - back;
            }
            accD += -fv * dv - dv * dv / (2.0 * lam * wv);
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
    const int grid = (int)std::min<int64_t>(nb, (int64_t)c->sm_count * 4);
    sweep_kernel<T><<<grid, kSweepThreads, 0, s>>>(a);
}

template <typename T>
void energy_t(denser_ctx* c, int64_t nb, cudaStream_t s) {
    const int cur = c->cur;
    energy_kernel<T><<<kEnergyGrid, kSweepThreads, 0, s>>>(
        (const T*)c->d.u, (const T*)c->d.p[cur], c->d.f, c->d.w, c->d.omega_bits, c->d.nbr,
        (size_t)c->d.max_blocks * kBlockVoxels, (int)nb, c->prm.lambda, c->d.partials);
    energy_final_kernel<<<1, 1024, 0, s>>>(c->d.partials, kEnergyGrid);
}

}  // namespace

int launch_prepare_regularize(denser_ctx* c, int64_t nb, bool rebuild_nbr, cudaStream_t s) {
    if (nb <= 0) return DENSER_OK;
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
