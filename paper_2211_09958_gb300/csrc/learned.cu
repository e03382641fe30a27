// Learned PM force correction: parameter packing, Adam, the loss residual
// and the density cotangent of the features.  The network's products run on
// the tensor cores (learned_tc.cu).
//
// The paper lists "spatiotemporal optimization of the PM gravity solver" as
// work built on pmwd (Statement of Need) without describing it; the network
// is this library's design:
//   features  asinh(rho(c + o) - 1) for the 27 periodic neighbour offsets o
//             (ox slowest, oz fastest), the scale factor a, 4 zeros (32)
//   network   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3
//             (32 -> 128 -> 128 -> 3)
//   output    dF_j(c) = s_out y_j(c), s_out = 3/2 Om h, added to the force
//             meshes before the CIC read
// Training matches forces: L = mean_i |read(dF)(x_i) - T_i|^2 with T the
// fine-mesh minus coarse-mesh PM force at the particles.

#include <cuda_bf16.h>

#include "pm_internal.h"

namespace pmgb {

namespace {

using bf16 = __nv_bfloat16;

constexpr int NI = NN_IN, NH = NN_HID, NO = NN_OUT;
constexpr int N3 = 16;  // padded output width of the tensor-core layer 3

// Flat FP32 parameters theta = [W1 32x128, b1, W2 128x128, b2, W3 128x3, b3]
// -> the packed bf16 operand copies and FP32 biases used by the kernels.
__global__ void k_nn_pack(const float *theta, NNWeightsMut w) {
    const float *W1 = theta, *b1 = W1 + NI * NH, *W2 = b1 + NH, *b2 = W2 + NH * NH, *W3 = b2 + NH, *b3 = W3 + NH * NO;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NH * NH; k += gridDim.x * blockDim.x) {
        // forward B operands, rows = outputs, K = inputs:
        //   w1c [128][32], w2c [128][128], w3c [16][128] (rows >= 3 zero)
        // backward B operands, rows = inputs, K = outputs:
        //   w2b [128][128], w3b [128][16] (K >= 3 zero), w1b [32][128]
        {
            const int r = k / NH, c = k % NH;
            w.w2c[nn_cm_index(r, c, NH)] = __float2bfloat16_rn(W2[c * NH + r]);
            w.w2b[nn_cm_index(r, c, NH)] = __float2bfloat16_rn(W2[r * NH + c]);
        }
        if (k < NH * NI) {
            const int r = k / NI, c = k % NI;  // hidden r, feature c
            w.w1c[nn_cm_index(r, c, NH)] = __float2bfloat16_rn(W1[c * NH + r]);
            const int f = k / NH, o = k % NH;  // feature f, hidden o
            w.w1b[nn_cm_index(f, o, NI)] = __float2bfloat16_rn(W1[f * NH + o]);
        }
        if (k < N3 * NH) {
            const int r = k / NH, c = k % NH;  // output r, hidden c
            w.w3c[nn_cm_index(r, c, N3)] = __float2bfloat16_rn(r < NO ? W3[c * NO + r] : 0.f);
            const int i = k / N3, o = k % N3;  // hidden i, output o
            w.w3b[nn_cm_index(i, o, NH)] = __float2bfloat16_rn(o < NO ? W3[i * NO + o] : 0.f);
        }
        if (k < NH) {
            w.b1[k] = b1[k];
            w.b2[k] = b2[k];
        }
        if (k < 8) w.b3[k] = k < NO ? b3[k] : 0.f;
    }
}

// Adam on the flat parameters (the gradient is left in place).
__global__ void k_adam(float *theta, float *grad, float *m, float *v, int np, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const float gk = grad[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk, vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        theta[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
    }
}

// Residual of the predicted per-particle correction against the target:
// loss += sum |pred - T|^2, pred <- 2 (pred - T) * scale (cotangent of
// weight * mean, scale = weight / n_particles).
__global__ void k_nn_residual(float *pred, const float *target, int64_t n, float scale, double *loss) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        acc += (double)d * d;
        pred[i] = 2.f * d * scale;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// g_rho(c) = sum_q g_x(c - o_q, q) / sqrt(1 + (rho(c) - 1)^2), divided by the
// run's kick factor (the read applies it to the whole VJP), into slot 3.
__global__ void k_nn_grad_rho(NNArgs a, const float *rho4, float *out4, int64_t cells) {
    const int n = a.n;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t run = c / n3, loc = c - run * n3;
        const int x = (int)(loc / ((int64_t)n * n)), y = (int)((loc / n) % n), z = (int)(loc % n);
        float acc = 0.f;
#pragma unroll 1
        for (int q = 0; q < 27; ++q) {
            const int ox = q / 9 - 1, oy = (q / 3) % 3 - 1, oz = q % 3 - 1;
            const int xx = (x - ox + n) % n, yy = (y - oy + n) % n, zz = (z - oz + n) % n;
            acc += a.gx[(run * n3 + ((int64_t)xx * n + yy) * n + zz) * NI + q];
        }
        const float r = rho4[c * 4] - 1.f;
        out4[c * 4 + 3] = acc * rsqrtf(1.f + r * r) / nn_kick_coef(a, run);
    }
}

__global__ void k_add4(float4 *dst, const float4 *src, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 s = src[i];
        float4 d = dst[i];
        d.x += s.x;
        d.y += s.y;
        d.z += s.z;
        d.w += s.w;
        dst[i] = d;
    }
}

}  // namespace

cudaError_t launch_nn_grad_rho(const NNArgs &a, const float *rho4, float *out4, int64_t cells, cudaStream_t st) {
    const int64_t blocks = (cells + 255) / 256;
    k_nn_grad_rho<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(a, rho4, out4, cells);
    return cudaGetLastError();
}

cudaError_t launch_add4(float4 *dst, const float4 *src, int64_t n, cudaStream_t st) {
    const int64_t blocks = (n + 255) / 256;
    k_add4<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(dst, src, n);
    return cudaGetLastError();
}

int nn_param_count() { return NI * NH + NH + NH * NH + NH + NH * NO + NO; }

size_t nn_packed_bytes() {
    return sizeof(bf16) * 2 * (NH * NI + NH * NH + N3 * NH) + sizeof(float) * (NH + NH + 8) + 16 * 9;
}

NNWeightsMut nn_carve(void *base) {
    NNWeightsMut w{};
    char *p = static_cast<char *>(base);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 15) / 16 * 16;
        return q;
    };
    w.w1c = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * NI));
    w.w2c = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * NH));
    w.w3c = reinterpret_cast<bf16 *>(take(sizeof(bf16) * N3 * NH));
    w.w1b = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NI * NH));
    w.w2b = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * NH));
    w.w3b = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * N3));
    w.b1 = reinterpret_cast<float *>(take(sizeof(float) * NH));
    w.b2 = reinterpret_cast<float *>(take(sizeof(float) * NH));
    w.b3 = reinterpret_cast<float *>(take(sizeof(float) * 8));
    return w;
}

cudaError_t launch_nn_pack(const float *theta, const NNWeightsMut &w, cudaStream_t st) {
    k_nn_pack<<<NH * NH / 256, 256, 0, st>>>(theta, w);
    return cudaGetLastError();
}

cudaError_t launch_nn_residual(float *pred, const float *target, int64_t n, float scale, double *loss,
                               cudaStream_t st) {
    const int64_t blocks = (n + 255) / 256;
    k_nn_residual<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(pred, target, n, scale, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *theta, float *grad, float *m, float *v, int np, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t st) {
    k_adam<<<(np + 255) / 256, 256, 0, st>>>(theta, grad, m, v, np, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace pmgb
