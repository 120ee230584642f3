// Depth-map estimation from a rectified stereo pair (Section IV): a Census Transform
// Signature data term (IV-A) and an affine TGV regulariser shaped by an image-driven
// diffusion tensor (IV-B, IV-C; weights from Table I).  Readings of what the paper
// leaves open, stated with the oracle as well:
//   * I_R is the reference image, rho(d, x, y) compares I_L(x + d, y) with I_R(x, y);
//   * 9 x 7 Census window (62 bits, row-major, centre skipped; a bit is set when that
//     neighbour is darker), edge pixels repeated; cost = Hamming / 62, 1 off the image;
//   * T = I + (exp(-gamma |grad I|^beta) - 1) n n^T, n = grad I / |grad I|, I where
//     grad I = 0 (forward differences of I_R);
//   * the data term is decoupled by an auxiliary field a: alternate an exhaustive
//     integer a-step, argmin_delta lam C + (d - delta)^2 / (2 theta) in float32 with a
//     fixed operation order (ties to the smaller delta), and a d-step of Chambolle-Pock
//     iterations on the TGV_T-L2 problem (duals p, |p| <= alpha1, and q, 2 x 2,
//     |q|_F <= alpha2; tau = sigma = 1/sqrt(12)), theta shrinking per outer step;
//   * forward differences, zero across the last column / row; div = -grad^T.
//
// Kernels: census, tensor, assign (one thread per pixel, the row's left signatures
// staged in shared memory), and one fused kernel per primal-dual iteration (the dual
// step on a tile and its halo in shared memory, then the primal step).  All buffers are
// device memory in planes of H x W floats (row-major).
#include "common.cuh"

namespace denser {

namespace {

constexpr int kRX = 4, kRY = 3;                         // 9 x 7 window
constexpr int kBits = (2 * kRX + 1) * (2 * kRY + 1) - 1;  // 62

__global__ void census_kernel(const float* __restrict__ I, int W, int H, unsigned long long* __restrict__ sig) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const float c = I[(size_t)y * W + x];
    unsigned long long s = 0;
    int b = 0;
#pragma unroll
    for (int dy = -kRY; dy <= kRY; ++dy) {
        const int yy = min(max(y + dy, 0), H - 1);
#pragma unroll
        for (int dx = -kRX; dx <= kRX; ++dx) {
            if (dx == 0 && dy == 0) continue;
            const int xx = min(max(x + dx, 0), W - 1);
            s |= (unsigned long long)(I[(size_t)yy * W + xx] < c ? 1u : 0u) << b;
            ++b;
        }
    }
    sig[(size_t)y * W + x] = s;
}

// T as three planes (t00, t01, t11).
__global__ void tensor_kernel(const float* __restrict__ I, int W, int H, float gamma, float beta,
                              float* __restrict__ T) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const size_t i = (size_t)y * W + x, n = (size_t)W * H;
    const float c = I[i];
    const float gx = x + 1 < W ? I[i + 1] - c : 0.0f;
    const float gy = y + 1 < H ? I[i + W] - c : 0.0f;
    const float mag = sqrtf(gx * gx + gy * gy);
    float t00 = 1.0f, t01 = 0.0f, t11 = 1.0f;
    if (mag > 0.0f) {
        const float em1 = expf(-gamma * powf(mag, beta)) - 1.0f;
        const float nx = gx / mag, ny = gy / mag;
        t00 = 1.0f + em1 * nx * nx;
        t01 = em1 * nx * ny;
        t11 = 1.0f + em1 * ny * ny;
    }
    T[i] = t00;
    T[n + i] = t01;
    T[2 * n + i] = t11;
}

// a-step.  CTA = 128 consecutive pixels of one row; the left signatures the row segment
// needs, x0 .. x0 + 127 + D - 1, sit in shared memory.  cq = 0 drops the coupling.
__global__ void __launch_bounds__(128) assign_kernel(const unsigned long long* __restrict__ sigL,
                                                     const unsigned long long* __restrict__ sigR, int W, int H, int D,
                                                     float cw, float cq, const float* __restrict__ d,
                                                     float* __restrict__ a) {
    extern __shared__ unsigned long long sl[];
    const int x0 = blockIdx.x * 128, y = blockIdx.y;
    const int span = min(128 + D - 1, W - x0);
    for (int i = threadIdx.x; i < span; i += 128) sl[i] = sigL[(size_t)y * W + x0 + i];
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    const unsigned long long r = sigR[i];
    const float dv = d[i];
    float best = __int_as_float(0x7f800000);  // +inf
    int arg = 0;
    for (int k = 0; k < D; ++k) {
        const int h = x + k < W ? __popcll(sl[threadIdx.x + k] ^ r) : kBits;
        const float dd = __fsub_rn(dv, (float)k);
        const float e = __fadd_rn(__fmul_rn((float)h, cw), __fmul_rn(__fmul_rn(dd, dd), cq));
        if (e < best) {
            best = e;
            arg = k;
        }
    }
    a[i] = (float)arg;
}

// State planes of the d-step.
enum Plane { kD = 0, kDb, kW1, kW2, kWb1, kWb2, kP1, kP2, kQ11, kQ12, kQ21, kQ22, kPlanes };

// (div v)(x, y) of a field v given at x - 1, x (for the x part) and y - 1, y.
__device__ __forceinline__ float div_x(int x, int W, float v, float vm) {
    return (x == 0 ? v : (x == W - 1 ? -vm : v - vm));
}

// One primal-dual iteration in one kernel.  A 32 x 8 tile stages d_bar and w_bar on
// its region plus a halo (-1 .. +1), takes the dual step on the tile and its -x / -y
// halo (the halo's duals are recomputed, identically, by the neighbouring tiles that
// own them), then the primal step on the tile.  Neighbours are read from Si and every
// plane written to So, so the call ping-pongs two state copies.
constexpr int kTX = 32, kTY = 8;
__global__ void __launch_bounds__(256) tgv_fused_kernel(const float* __restrict__ Si, float* __restrict__ So,
                                                        const float* __restrict__ T, const float* __restrict__ a,
                                                        int W, int H, float sigma, float tau, float tau_theta,
                                                        float alpha1, float alpha2) {
    __shared__ float sdb[kTY + 2][kTX + 2], sw1[kTY + 2][kTX + 2], sw2[kTY + 2][kTX + 2];
    __shared__ float st0[kTY + 1][kTX + 1], st1[kTY + 1][kTX + 1], st2[kTY + 1][kTX + 1];
    __shared__ float sp1[kTY + 1][kTX + 1], sp2[kTY + 1][kTX + 1];
    __shared__ float sq11[kTY + 1][kTX + 1], sq12[kTY + 1][kTX + 1], sq21[kTY + 1][kTX + 1], sq22[kTY + 1][kTX + 1];
    const size_t n = (size_t)W * H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, tid = threadIdx.x;
    // d_bar, w_bar on [x0 - 1, x0 + kTX] x [y0 - 1, y0 + kTY]
    for (int k = tid; k < (kTY + 2) * (kTX + 2); k += 256) {
        const int ry = k / (kTX + 2), rx = k % (kTX + 2);
        const int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
        float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const size_t i = (size_t)gy * W + gx;
            v0 = Si[kDb * n + i], v1 = Si[kWb1 * n + i], v2 = Si[kWb2 * n + i];
        }
        sdb[ry][rx] = v0, sw1[ry][rx] = v1, sw2[ry][rx] = v2;
    }
    __syncthreads();
    // dual step on [x0 - 1, x0 + kTX - 1] x [y0 - 1, y0 + kTY - 1]
    for (int k = tid; k < (kTY + 1) * (kTX + 1); k += 256) {
        const int ry = k / (kTX + 1), rx = k % (kTX + 1);
        const int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
        float t0 = 1.0f, t1 = 0.0f, t2 = 1.0f, p1 = 0.0f, p2 = 0.0f, q11 = 0.0f, q12 = 0.0f, q21 = 0.0f, q22 = 0.0f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const size_t i = (size_t)gy * W + gx;
            const bool hx = gx + 1 < W, hy = gy + 1 < H;
            const float db = sdb[ry][rx];
            const float gxd = hx ? sdb[ry][rx + 1] - db : 0.0f, gyd = hy ? sdb[ry + 1][rx] - db : 0.0f;
            t0 = T[i], t1 = T[n + i], t2 = T[2 * n + i];
            p1 = Si[kP1 * n + i] + sigma * ((t0 * gxd + t1 * gyd) - sw1[ry][rx]);
            p2 = Si[kP2 * n + i] + sigma * ((t1 * gxd + t2 * gyd) - sw2[ry][rx]);
            const float sp = fmaxf(1.0f, sqrtf(p1 * p1 + p2 * p2) / alpha1);
            p1 /= sp, p2 /= sp;
            const float w1 = sw1[ry][rx], w2 = sw2[ry][rx];
            const float g11 = hx ? sw1[ry][rx + 1] - w1 : 0.0f, g12 = hy ? sw1[ry + 1][rx] - w1 : 0.0f;
            const float g21 = hx ? sw2[ry][rx + 1] - w2 : 0.0f, g22 = hy ? sw2[ry + 1][rx] - w2 : 0.0f;
            q11 = Si[kQ11 * n + i] + sigma * g11, q12 = Si[kQ12 * n + i] + sigma * g12;
            q21 = Si[kQ21 * n + i] + sigma * g21, q22 = Si[kQ22 * n + i] + sigma * g22;
            const float sq = fmaxf(1.0f, sqrtf(q11 * q11 + q12 * q12 + q21 * q21 + q22 * q22) / alpha2);
            q11 /= sq, q12 /= sq, q21 /= sq, q22 /= sq;
        }
        st0[ry][rx] = t0, st1[ry][rx] = t1, st2[ry][rx] = t2;
        sp1[ry][rx] = p1, sp2[ry][rx] = p2;
        sq11[ry][rx] = q11, sq12[ry][rx] = q12, sq21[ry][rx] = q21, sq22[ry][rx] = q22;
    }
    __syncthreads();
    // primal step on the tile
    const int rx = (tid & (kTX - 1)) + 1, ry = tid / kTX + 1;
    const int gx = x0 + rx - 1, gy = y0 + ry - 1;
    if (gx >= W || gy >= H) return;
    const size_t i = (size_t)gy * W + gx;
    const float tp1 = st0[ry][rx] * sp1[ry][rx] + st1[ry][rx] * sp2[ry][rx];
    const float tp2 = st1[ry][rx] * sp1[ry][rx] + st2[ry][rx] * sp2[ry][rx];
    const float tp1m = gx > 0 ? st0[ry][rx - 1] * sp1[ry][rx - 1] + st1[ry][rx - 1] * sp2[ry][rx - 1] : 0.0f;
    const float tp2m = gy > 0 ? st1[ry - 1][rx] * sp1[ry - 1][rx] + st2[ry - 1][rx] * sp2[ry - 1][rx] : 0.0f;
    const float divTp = div_x(gx, W, tp1, tp1m) + div_x(gy, H, tp2, tp2m);
    const float d_old = Si[kD * n + i];
    const float d_new = (d_old + tau * divTp + tau_theta * a[i]) / (1.0f + tau_theta);
    const float dq1 = div_x(gx, W, sq11[ry][rx], gx > 0 ? sq11[ry][rx - 1] : 0.0f) +
                      div_x(gy, H, sq12[ry][rx], gy > 0 ? sq12[ry - 1][rx] : 0.0f);
    const float dq2 = div_x(gx, W, sq21[ry][rx], gx > 0 ? sq21[ry][rx - 1] : 0.0f) +
                      div_x(gy, H, sq22[ry][rx], gy > 0 ? sq22[ry - 1][rx] : 0.0f);
    const float w1o = Si[kW1 * n + i], w2o = Si[kW2 * n + i];
    const float w1 = w1o + tau * (sp1[ry][rx] + dq1), w2 = w2o + tau * (sp2[ry][rx] + dq2);
    So[kD * n + i] = d_new;
    So[kDb * n + i] = 2.0f * d_new - d_old;
    So[kW1 * n + i] = w1;
    So[kW2 * n + i] = w2;
    So[kWb1 * n + i] = 2.0f * w1 - w1o;
    So[kWb2 * n + i] = 2.0f * w2 - w2o;
    So[kP1 * n + i] = sp1[ry][rx];
    So[kP2 * n + i] = sp2[ry][rx];
    So[kQ11 * n + i] = sq11[ry][rx];
    So[kQ12 * n + i] = sq12[ry][rx];
    So[kQ21 * n + i] = sq21[ry][rx];
    So[kQ22 * n + i] = sq22[ry][rx];
}

__global__ void init_state_kernel(float* __restrict__ S, const float* __restrict__ d0, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        S[kD * n + i] = d0[i];
        S[kDb * n + i] = d0[i];
        for (int k = kW1; k < kPlanes; ++k) S[k * n + i] = 0.0f;
    }
}

__global__ void depth_kernel(const float* __restrict__ disp, size_t n, float fb, float min_disp,
                             float* __restrict__ depth) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float dv = disp[i];
        depth[i] = dv > min_disp ? fb / dv : 0.0f;
    }
}

}  // namespace

int stereo_census(const float* img, int W, int H, unsigned long long* sig, cudaStream_t s) {
    census_kernel<<<dim3((W + 127) / 128, H), 128, 0, s>>>(img, W, H, sig);
    return cudaGetLastError() == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

int stereo_tensor(const float* img, int W, int H, float gamma, float beta, float* T, cudaStream_t s) {
    tensor_kernel<<<dim3((W + 127) / 128, H), 128, 0, s>>>(img, W, H, gamma, beta, T);
    return cudaGetLastError() == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

int stereo_assign(const unsigned long long* sigL, const unsigned long long* sigR, int W, int H, int D, float lambda,
                  double theta, const float* d, float* a, cudaStream_t s) {
    const float cw = (float)(lambda / kBits);
    const float cq = (theta > 0 && isfinite(theta)) ? (float)(1.0 / (2.0 * theta)) : 0.0f;
    const size_t smem = (size_t)(128 + D) * 8;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return DENSER_ERR_CUDA;
    }
    assign_kernel<<<dim3((W + 127) / 128, H), 128, smem, s>>>(sigL, sigR, W, H, D, cw, cq, d, a);
    return cudaGetLastError() == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

// state: 2 x 12 planes; the first copy holds the state on entry and on return, the
// second is the ping-pong partner of the fused kernel.
int stereo_tgv(const float* a, const float* T, int W, int H, float alpha1, float alpha2, double theta, int iters,
               float* state, cudaStream_t s) {
    const float tau = (float)(1.0 / sqrt(12.0));
    const size_t plane = (size_t)W * H;
    float* A = state;
    float* B = state + kPlanes * plane;
    const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY);
    for (int k = 0; k < iters; ++k) {
        const bool even = (k & 1) == 0;
        tgv_fused_kernel<<<grid, 256, 0, s>>>(even ? A : B, even ? B : A, T, a, W, H, tau, tau, (float)(tau / theta),
                                              alpha1, alpha2);
    }
    if (iters & 1) {
        if (cudaMemcpyAsync(A, B, kPlanes * plane * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return DENSER_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

int stereo_init_state(float* state, const float* d0, int W, int H, cudaStream_t s) {
    const size_t n = (size_t)W * H;
    init_state_kernel<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(state, d0, n);
    return cudaGetLastError() == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

int stereo_depth(const float* disp, int W, int H, float fb, float min_disp, float* depth, cudaStream_t s) {
    const size_t n = (size_t)W * H;
    depth_kernel<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(disp, n, fb, min_disp, depth);
    return cudaGetLastError() == cudaSuccess ? DENSER_OK : DENSER_ERR_CUDA;
}

}  // namespace denser
