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
// staged in shared memory), and per primal-dual iteration a dual kernel (p, q) and a
// primal kernel (d, w and their over-relaxed copies).  All buffers are device memory
// in planes of H x W floats (row-major).
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

// Dual step: p <- P_alpha1(p + sigma (T grad d_bar - w_bar)), q <- P_alpha2(q + sigma grad w_bar).
__global__ void tgv_dual_kernel(float* __restrict__ S, const float* __restrict__ T, int W, int H, float sigma,
                                float alpha1, float alpha2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const size_t n = (size_t)W * H, i = (size_t)y * W + x;
    const bool hx = x + 1 < W, hy = y + 1 < H;
    const float* db = S + kDb * n;
    const float* wb1 = S + kWb1 * n;
    const float* wb2 = S + kWb2 * n;
    const float gx = hx ? db[i + 1] - db[i] : 0.0f, gy = hy ? db[i + W] - db[i] : 0.0f;
    const float t00 = T[i], t01 = T[n + i], t11 = T[2 * n + i];
    float p1 = S[kP1 * n + i] + sigma * ((t00 * gx + t01 * gy) - wb1[i]);
    float p2 = S[kP2 * n + i] + sigma * ((t01 * gx + t11 * gy) - wb2[i]);
    const float sp = fmaxf(1.0f, sqrtf(p1 * p1 + p2 * p2) / alpha1);
    S[kP1 * n + i] = p1 / sp;
    S[kP2 * n + i] = p2 / sp;
    const float g11 = hx ? wb1[i + 1] - wb1[i] : 0.0f, g12 = hy ? wb1[i + W] - wb1[i] : 0.0f;
    const float g21 = hx ? wb2[i + 1] - wb2[i] : 0.0f, g22 = hy ? wb2[i + W] - wb2[i] : 0.0f;
    float q11 = S[kQ11 * n + i] + sigma * g11, q12 = S[kQ12 * n + i] + sigma * g12;
    float q21 = S[kQ21 * n + i] + sigma * g21, q22 = S[kQ22 * n + i] + sigma * g22;
    const float sq = fmaxf(1.0f, sqrtf(q11 * q11 + q12 * q12 + q21 * q21 + q22 * q22) / alpha2);
    S[kQ11 * n + i] = q11 / sq;
    S[kQ12 * n + i] = q12 / sq;
    S[kQ21 * n + i] = q21 / sq;
    S[kQ22 * n + i] = q22 / sq;
}

// (div v)(x, y) of a field v given at x - 1, x (for the x part) and y - 1, y.
__device__ __forceinline__ float div_x(int x, int W, float v, float vm) {
    return (x == 0 ? v : (x == W - 1 ? -vm : v - vm));
}

// Primal step: d <- prox(d + tau div(T p)), w <- w + tau (p + div q); over-relaxation.
__global__ void tgv_primal_kernel(float* __restrict__ S, const float* __restrict__ T, const float* __restrict__ a,
                                  int W, int H, float tau, float tau_theta) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const size_t n = (size_t)W * H, i = (size_t)y * W + x;
    const float* P1 = S + kP1 * n;
    const float* P2 = S + kP2 * n;
    // T p at the pixel and its -x, -y neighbours (T is symmetric)
    const float tp1 = T[i] * P1[i] + T[n + i] * P2[i];
    const float tp2 = T[n + i] * P1[i] + T[2 * n + i] * P2[i];
    float tp1m = 0.0f, tp2m = 0.0f;
    if (x > 0) tp1m = T[i - 1] * P1[i - 1] + T[n + i - 1] * P2[i - 1];
    if (y > 0) tp2m = T[n + i - W] * P1[i - W] + T[2 * n + i - W] * P2[i - W];
    const float divTp = div_x(x, W, tp1, tp1m) + div_x(y, H, tp2, tp2m);
    const float d_old = S[kD * n + i];
    const float d_new = (d_old + tau * divTp + tau_theta * a[i]) / (1.0f + tau_theta);
    // div q per component (q[i][0] pairs with d/dx, q[i][1] with d/dy)
    const float* Q11 = S + kQ11 * n;
    const float* Q12 = S + kQ12 * n;
    const float* Q21 = S + kQ21 * n;
    const float* Q22 = S + kQ22 * n;
    const float dq1 = div_x(x, W, Q11[i], x > 0 ? Q11[i - 1] : 0.0f) + div_x(y, H, Q12[i], y > 0 ? Q12[i - W] : 0.0f);
    const float dq2 = div_x(x, W, Q21[i], x > 0 ? Q21[i - 1] : 0.0f) + div_x(y, H, Q22[i], y > 0 ? Q22[i - W] : 0.0f);
    const float w1o = S[kW1 * n + i], w2o = S[kW2 * n + i];
    const float w1 = w1o + tau * (P1[i] + dq1), w2 = w2o + tau * (P2[i] + dq2);
    S[kD * n + i] = d_new;
    S[kDb * n + i] = 2.0f * d_new - d_old;
    S[kW1 * n + i] = w1;
    S[kW2 * n + i] = w2;
    S[kWb1 * n + i] = 2.0f * w1 - w1o;
    S[kWb2 * n + i] = 2.0f * w2 - w2o;
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

int stereo_tgv(const float* a, const float* T, int W, int H, float alpha1, float alpha2, double theta, int iters,
               float* state, cudaStream_t s) {
    const float tau = (float)(1.0 / sqrt(12.0));
    const dim3 grid((W + 127) / 128, H);
    for (int k = 0; k < iters; ++k) {
        tgv_dual_kernel<<<grid, 128, 0, s>>>(state, T, W, H, tau, alpha1, alpha2);
        tgv_primal_kernel<<<grid, 128, 0, s>>>(state, T, a, W, H, tau, (float)(tau / theta));
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
