// Learned PM force correction: a per-cell MLP on the coarse CIC density,
// BF16 tensor-core products (mma.sync m16n8k16) accumulating in FP32.
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
//
// Fragment layouts of mma.m16n8k16 (lane = 4 g + t):
//   A (16x16, row): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..],
//                   a3 = A[g+8][2t+8..]
//   B (16x8, col):  b0 = B[2t..2t+1][g], b1 = B[2t+8..2t+9][g]
//   C (16x8):       c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t],
//                   c3 = C[g+8][2t+1]
// Two adjacent 8-column C tiles are exactly one 16-column A tile, so each
// layer's output feeds the next product without leaving registers.

#include <cuda_bf16.h>

#include "pm_internal.h"

namespace pmgb {

namespace {

using bf16 = __nv_bfloat16;

constexpr int NI = NN_IN, NH = NN_HID, NO = NN_OUT;
constexpr int KP1 = NI + 8;  // padded row (bf16) of 32-wide operands
constexpr int KP2 = NH + 8;  // padded row of 128-wide operands
constexpr int KP3 = 24;      // padded row of 16-wide operands
constexpr int TILE = 128;    // cells per block
constexpr int THREADS = 256;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_bf(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ float2 unpack2(uint32_t u) {
    __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&u);
    return __bfloat1622float2(v);
}

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Copy n16 16-byte chunks from global to shared memory.
__device__ __forceinline__ void copy16(void *dst, const void *src, int n16) {
    for (int k = threadIdx.x; k < n16; k += blockDim.x)
        reinterpret_cast<int4 *>(dst)[k] = reinterpret_cast<const int4 *>(src)[k];
}

// Layer product C[16 x 8 J] += A[16 x 16 KK] B with A as register fragments
// and B from shared memory rows of length ld (B col-major: row n holds K).
template <int KK, int J>
__device__ __forceinline__ void layer(float (&acc)[J][4], const uint32_t (&af)[KK][4], const bf16 *bs, int ld, int g,
                                      int t) {
#pragma unroll
    for (int kk = 0; kk < KK; ++kk)
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const bf16 *row = bs + (8 * j + g) * ld + 16 * kk + 2 * t;
            mma(acc[j], af[kk], ld32(row), ld32(row + 8));
        }
}

// Bias + ReLU of a [16 x 128] accumulator, packed into A fragments.
__device__ __forceinline__ void relu_pack(float (&acc)[NH / 8][4], const float *bias, uint32_t (&af)[NH / 16][4],
                                          int t) {
#pragma unroll
    for (int j = 0; j < NH / 8; ++j) {
        const float bx = bias[8 * j + 2 * t], by = bias[8 * j + 2 * t + 1];
        const float v0 = fmaxf(acc[j][0] + bx, 0.f), v1 = fmaxf(acc[j][1] + by, 0.f);
        const float v2 = fmaxf(acc[j][2] + bx, 0.f), v3 = fmaxf(acc[j][3] + by, 0.f);
        af[j >> 1][(j & 1) * 2] = pack2(v0, v1);
        af[j >> 1][(j & 1) * 2 + 1] = pack2(v2, v3);
    }
}

// Store A fragments of a [16 x 128] activation tile to rows r0.. of a
// row-major global [cells][128] bf16 array.
__device__ __forceinline__ void store_frags(bf16 *dst, int64_t r0, const uint32_t (&af)[NH / 16][4], int g, int t) {
#pragma unroll
    for (int kk = 0; kk < NH / 16; ++kk) {
        const int c = 16 * kk + 2 * t;
        *reinterpret_cast<uint32_t *>(dst + (r0 + g) * NH + c) = af[kk][0];
        *reinterpret_cast<uint32_t *>(dst + (r0 + g + 8) * NH + c) = af[kk][1];
        *reinterpret_cast<uint32_t *>(dst + (r0 + g) * NH + c + 8) = af[kk][2];
        *reinterpret_cast<uint32_t *>(dst + (r0 + g + 8) * NH + c + 8) = af[kk][3];
    }
}

struct SmemFwd {
    static constexpr int X = TILE * KP1, W1 = NH * KP1, W2 = NH * KP2, W3 = 8 * KP2;
    static constexpr size_t BYTES = sizeof(bf16) * (X + W1 + W2 + W3) + sizeof(float) * (NH + NH + 8);
};

// Inference (and the training forward), persistent: each block stages the
// weights once and walks tiles of 128 cells (one run per tile, n^3 is a
// multiple of 128); warp w owns cells 16w .. 16w + 15 of a tile.
template <bool TRAIN>
__global__ void __launch_bounds__(THREADS, 2) k_mlp_fwd(NNArgs a, int64_t tiles) {
    extern __shared__ int4 smraw[];
    bf16 *Xs = reinterpret_cast<bf16 *>(smraw);
    bf16 *W1s = Xs + SmemFwd::X, *W2s = W1s + SmemFwd::W1, *W3s = W2s + SmemFwd::W2;
    float *bs = reinterpret_cast<float *>(W3s + SmemFwd::W3);
    copy16(W1s, a.w.w1t, SmemFwd::W1 * 2 / 16);
    copy16(W2s, a.w.w2t, SmemFwd::W2 * 2 / 16);
    copy16(W3s, a.w.w3t, SmemFwd::W3 * 2 / 16);
    copy16(bs, a.w.b1, NH * 4 / 16);
    copy16(bs + NH, a.w.b2, NH * 4 / 16);
    copy16(bs + 2 * NH, a.w.b3, 8 * 4 / 16);

    const int n = a.n;
    const int64_t n3 = (int64_t)n * n * n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = 16 * warp;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t cell0 = tile * TILE;  // global cell index (run-major)
    const int64_t run = cell0 / n3;
    const int rs = a.rho_stride == 4 ? 4 : 1;
    const float *rho = a.rho + run * n3 * rs;
    const float s_out = a.pref[run] * a.s_scale;
    __syncthreads();  // previous tile's feature rows are consumed
    {
        const int cl = threadIdx.x & (TILE - 1), half = threadIdx.x >> 7;
        const int64_t c = cell0 - run * n3 + cl;
        const int x = (int)(c / ((int64_t)n * n)), y = (int)((c / n) % n), z = (int)(c % n);
        bf16 *row = Xs + cl * KP1;
        for (int q = half ? 14 : 0; q < (half ? 27 : 14); ++q) {
            const int ox = q / 9 - 1, oy = (q / 3) % 3 - 1, oz = q % 3 - 1;
            const int xx = (x + ox + n) % n, yy = (y + oy + n) % n, zz = (z + oz + n) % n;
            const float v = __ldg(rho + (((int64_t)xx * n + yy) * n + zz) * rs);
            row[q] = __float2bfloat16_rn(asinhf(v - 1.f));
        }
        if (half) {
            row[27] = __float2bfloat16_rn(a.afeat);
            for (int q = 28; q < KP1; ++q) row[q] = __float2bfloat16_rn(0.f);
        }
    }
    __syncthreads();
    if (TRAIN) {  // features, for the first layer's weight gradient
        const bf16 *src = Xs + (m0 + g) * KP1;
        for (int k = t; k < NI / 2; k += 4) {
            *reinterpret_cast<uint32_t *>(a.xg + (cell0 + m0 + g) * NI + 2 * k) = ld32(src + 2 * k);
            *reinterpret_cast<uint32_t *>(a.xg + (cell0 + m0 + g + 8) * NI + 2 * k) = ld32(src + 8 * KP1 + 2 * k);
        }
    }
    uint32_t xf[NI / 16][4];
#pragma unroll
    for (int kk = 0; kk < NI / 16; ++kk) {
        const bf16 *r0 = Xs + (m0 + g) * KP1 + 16 * kk + 2 * t;
        xf[kk][0] = ld32(r0);
        xf[kk][1] = ld32(r0 + 8 * KP1);
        xf[kk][2] = ld32(r0 + 8);
        xf[kk][3] = ld32(r0 + 8 * KP1 + 8);
    }
    float acc[NH / 8][4];
    uint32_t h[NH / 16][4];
#pragma unroll
    for (int j = 0; j < NH / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    layer<NI / 16, NH / 8>(acc, xf, W1s, KP1, g, t);
    relu_pack(acc, bs, h, t);
    if (TRAIN) store_frags(a.h1g, cell0 + m0, h, g, t);
#pragma unroll
    for (int j = 0; j < NH / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    layer<NH / 16, NH / 8>(acc, h, W2s, KP2, g, t);
    relu_pack(acc, bs + NH, h, t);
    if (TRAIN) store_frags(a.h2g, cell0 + m0, h, g, t);
    float o[1][4] = {{0.f, 0.f, 0.f, 0.f}};
    layer<NH / 16, 1>(o, h, W3s, KP2, g, t);
    // outputs j = 2t, 2t + 1 of cells m0 + g and m0 + g + 8
    const float *b3 = bs + 2 * NH;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int j = 2 * t + (e & 1);
        if (j >= NO) continue;
        const int64_t cell = cell0 + m0 + g + (e >> 1) * 8;
        float *dst = a.out + cell * 4 + j;
        const float v = s_out * (o[0][e] + b3[j]);
        if (a.accumulate)
            *dst += v;
        else
            *dst = v;
    }
    }
}

struct SmemBwd {
    static constexpr int W2 = NH * KP2, W3 = NH * KP3, W1 = NI * KP2;
    static constexpr size_t BYTES = sizeof(bf16) * (W2 + W3 + W1) + sizeof(float) * (2 * NH + 8);
};

__device__ __forceinline__ float kick_coef(const NNArgs &a, int64_t run) {
    if (!a.table) return 1.f;
    const float4 t = a.table[(int64_t)a.kick_step * a.nb + run];
    return a.kick_sel == KICK_A ? t.x : (a.kick_sel == KICK_B ? t.z : t.w);
}

// Backward through the network for 128 cells per block: from the output
// cotangent (slots 1..3 of the interleaved gradient mesh, times s_out) to the
// activation cotangents g2, g1 (stored as bf16), with the bias gradients.
__global__ void __launch_bounds__(THREADS, 2) k_mlp_bwd(NNArgs a, int64_t tiles) {
    extern __shared__ int4 smraw[];
    bf16 *W2n = reinterpret_cast<bf16 *>(smraw), *W3n = W2n + SmemBwd::W2, *W1n = W3n + SmemBwd::W3;
    float *gbs = reinterpret_cast<float *>(W1n + SmemBwd::W1);  // block sums of gb2 [128], gb1 [128], gb3 [8]
    copy16(W2n, a.w.w2n, SmemBwd::W2 * 2 / 16);
    copy16(W3n, a.w.w3n, SmemBwd::W3 * 2 / 16);
    if (a.gx) copy16(W1n, a.w.w1n, SmemBwd::W1 * 2 / 16);
    for (int k = threadIdx.x; k < 2 * NH + 8; k += THREADS) gbs[k] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t n3 = (int64_t)a.n * a.n * a.n;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t r0 = tile * TILE + 16 * warp;
    const float s_out = a.pref[tile * TILE / n3] * a.s_scale * kick_coef(a, tile * TILE / n3);
    // output cotangent, C layout [16 x 8]; columns >= 3 are zero
    float gy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int j = 2 * t + (e & 1);
        const int64_t cell = r0 + g + (e >> 1) * 8;
        const float v = j < NO ? s_out * a.gmesh[cell * 4 + 1 + j] : 0.f;
        gy[e] = __bfloat162float(__float2bfloat16_rn(v));
    }
    // bias gradient of layer 3 and the stored bf16 cotangent
    {
        float s0 = gy[0] + gy[2], s1 = gy[1] + gy[3];
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (g == 0) {
            atomicAdd(gbs + 2 * NH + 2 * t, s0);
            atomicAdd(gbs + 2 * NH + 2 * t + 1, s1);
        }
        *reinterpret_cast<uint32_t *>(a.g3g + (r0 + g) * 8 + 2 * t) = pack2(gy[0], gy[1]);
        *reinterpret_cast<uint32_t *>(a.g3g + (r0 + g + 8) * 8 + 2 * t) = pack2(gy[2], gy[3]);
    }
    uint32_t gf3[1][4] = {{pack2(gy[0], gy[1]), pack2(gy[2], gy[3]), 0u, 0u}};
    float acc[NH / 8][4];
    uint32_t gf[NH / 16][4];
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: g2 = (gy W3^T) * [h2 > 0]; pass 1: g1 = (g2 W2^T) * [h1 > 0]
#pragma unroll
        for (int j = 0; j < NH / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        if (pass == 0)
            layer<1, NH / 8>(acc, gf3, W3n, KP3, g, t);
        else
            layer<NH / 16, NH / 8>(acc, gf, W2n, KP2, g, t);
        const bf16 *hg = pass == 0 ? a.h2g : a.h1g;
        float *gb = gbs + pass * NH;
        bf16 *dst = pass == 0 ? a.g2g : a.g1g;
#pragma unroll
        for (int j = 0; j < NH / 8; ++j) {
            const int c = 8 * j + 2 * t;
            const float2 hA = unpack2(ld32(hg + (r0 + g) * NH + c));
            const float2 hB = unpack2(ld32(hg + (r0 + g + 8) * NH + c));
            const float v0 = hA.x > 0.f ? acc[j][0] : 0.f, v1 = hA.y > 0.f ? acc[j][1] : 0.f;
            const float v2 = hB.x > 0.f ? acc[j][2] : 0.f, v3 = hB.y > 0.f ? acc[j][3] : 0.f;
            float s0 = v0 + v2, s1 = v1 + v3;
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (g == 0) {
                atomicAdd(gb + c, s0);
                atomicAdd(gb + c + 1, s1);
            }
            gf[j >> 1][(j & 1) * 2] = pack2(v0, v1);
            gf[j >> 1][(j & 1) * 2 + 1] = pack2(v2, v3);
        }
        store_frags(dst, r0, gf, g, t);
    }
    if (a.gx) {
        // feature cotangent g_x = g1 W1^T (rows r0 .. r0 + 15, 32 features)
        float ax[NI / 8][4];
#pragma unroll
        for (int j = 0; j < NI / 8; ++j) ax[j][0] = ax[j][1] = ax[j][2] = ax[j][3] = 0.f;
        layer<NH / 16, NI / 8>(ax, gf, W1n, KP2, g, t);
#pragma unroll
        for (int j = 0; j < NI / 8; ++j) {
            const int c = 8 * j + 2 * t;
            *reinterpret_cast<float2 *>(a.gx + (r0 + g) * NI + c) = make_float2(ax[j][0], ax[j][1]);
            *reinterpret_cast<float2 *>(a.gx + (r0 + g + 8) * NI + c) = make_float2(ax[j][2], ax[j][3]);
        }
    }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * NH + NO; k += THREADS) {
        float *dst = k < NH ? a.gb2 + k : (k < 2 * NH ? a.gb1 + (k - NH) : a.gb3 + (k - 2 * NH));
        atomicAdd(dst, gbs[k]);
    }
}

// Weight gradient dW[K1][N] += sum over cells of A[c][i] B[c][j]
// (A: [cells][K1] activations, B: [cells][LB] cotangents), reduced over
// chunks of 128 cells per block, accumulated in registers, added to the
// global FP32 gradient (row pitch ldo, columns < nvalid) at the end.
template <int K1, int N, int LB>
__global__ void __launch_bounds__(THREADS) k_wgrad(const bf16 *__restrict__ A, const bf16 *__restrict__ B,
                                                   int64_t cells, float *out, int ldo, int nvalid) {
    constexpr int LA = K1 + 8, LBP = LB + 8;
    constexpr int MT = K1 / 16, NT = N / 8;           // dW tiles
    constexpr int TPW = MT * NT / 8;                  // tiles per warp
    constexpr int NPW = TPW < NT ? TPW : NT;          // n tiles per warp
    extern __shared__ int4 smraw[];
    bf16 *As = reinterpret_cast<bf16 *>(smraw), *Bs = As + TILE * LA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int mt = (warp * TPW) / NT, nt0 = (warp * TPW) % NT;
    float acc[NPW][4];
#pragma unroll
    for (int j = 0; j < NPW; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int64_t chunks = cells / TILE;
    for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        __syncthreads();
        const bf16 *ga = A + ch * TILE * K1, *gb = B + ch * TILE * LB;
        for (int k = threadIdx.x; k < TILE * K1 / 2; k += THREADS) {
            const int r = (2 * k) / K1, c = (2 * k) % K1;
            *reinterpret_cast<uint32_t *>(As + r * LA + c) = ld32(ga + 2 * k);
        }
        for (int k = threadIdx.x; k < TILE * LB / 2; k += THREADS) {
            const int r = (2 * k) / LB, c = (2 * k) % LB;
            *reinterpret_cast<uint32_t *>(Bs + r * LBP + c) = ld32(gb + 2 * k);
        }
        __syncthreads();
#pragma unroll
        for (int kc = 0; kc < TILE / 16; ++kc) {
            const int c0 = 16 * kc + 2 * t;
            const int i0 = 16 * mt + g;
            uint32_t af[4];
            af[0] = pack_bf(As[c0 * LA + i0], As[(c0 + 1) * LA + i0]);
            af[1] = pack_bf(As[c0 * LA + i0 + 8], As[(c0 + 1) * LA + i0 + 8]);
            af[2] = pack_bf(As[(c0 + 8) * LA + i0], As[(c0 + 9) * LA + i0]);
            af[3] = pack_bf(As[(c0 + 8) * LA + i0 + 8], As[(c0 + 9) * LA + i0 + 8]);
#pragma unroll
            for (int j = 0; j < NPW; ++j) {
                const int jn = 8 * (nt0 + j) + g;
                const uint32_t b0 = pack_bf(Bs[c0 * LBP + jn], Bs[(c0 + 1) * LBP + jn]);
                const uint32_t b1 = pack_bf(Bs[(c0 + 8) * LBP + jn], Bs[(c0 + 9) * LBP + jn]);
                mma(acc[j], af, b0, b1);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NPW; ++j) {
        const int i = 16 * mt + g, c = 8 * (nt0 + j) + 2 * t;
        if (c < nvalid) {
            atomicAdd(out + i * ldo + c, acc[j][0]);
            atomicAdd(out + (i + 8) * ldo + c, acc[j][2]);
        }
        if (c + 1 < nvalid) {
            atomicAdd(out + i * ldo + c + 1, acc[j][1]);
            atomicAdd(out + (i + 8) * ldo + c + 1, acc[j][3]);
        }
    }
}

// Flat FP32 parameters theta = [W1 32x128, b1, W2 128x128, b2, W3 128x3, b3]
// -> the packed bf16 operand copies and FP32 biases used by the kernels.
__global__ void k_nn_pack(const float *theta, NNWeightsMut w) {
    const float *W1 = theta, *b1 = W1 + NI * NH, *W2 = b1 + NH, *b2 = W2 + NH * NH, *W3 = b2 + NH, *b3 = W3 + NH * NO;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NH * KP2; k += gridDim.x * blockDim.x) {
        const int r = k / KP2, c = k % KP2;  // NH * KP2 > NH * NH: every index below is reached
        w.w2t[k] = __float2bfloat16_rn(c < NH ? W2[c * NH + r] : 0.f);  // [out][in]
        w.w2n[k] = __float2bfloat16_rn(c < NH ? W2[r * NH + c] : 0.f);  // [in][out]
        if (k < NH * KP1) {
            const int r1 = k / KP1, c1 = k % KP1;
            w.w1t[k] = __float2bfloat16_rn(c1 < NI ? W1[c1 * NH + r1] : 0.f);
        }
        if (k < 8 * KP2) w.w3t[k] = __float2bfloat16_rn(r < NO && c < NH ? W3[c * NO + r] : 0.f);
        if (k < NH * KP3) {
            const int r3 = k / KP3, c3 = k % KP3;
            w.w3n[k] = __float2bfloat16_rn(c3 < NO ? W3[r3 * NO + c3] : 0.f);
        }
        if (k < NI * KP2) {
            const int rn = k / KP2, cn = k % KP2;  // [feature][hidden]
            w.w1n[k] = __float2bfloat16_rn(cn < NH ? W1[rn * NH + cn] : 0.f);
        }
        if (k < NH) {
            w.b1[k] = b1[k];
            w.b2[k] = b2[k];
        }
        if (k < 8) w.b3[k] = k < NO ? b3[k] : 0.f;
        // tcgen05 operands: rows = outputs, K = inputs, core-matrix layout
        {
            const int r = k / NH, c = k % NH;  // k < NH * NH covers W2
            if (k < NH * NH) w.w2c[nn_cm_index(r, c, NH)] = __float2bfloat16_rn(W2[c * NH + r]);
            if (k < NH * NI) {
                const int r1 = k / NI, c1 = k % NI;
                w.w1c[nn_cm_index(r1, c1, NH)] = __float2bfloat16_rn(W1[c1 * NH + r1]);
            }
            if (k < 16 * NH) {
                const int r3 = k / NH, c3 = k % NH;
                w.w3c[nn_cm_index(r3, c3, 16)] = __float2bfloat16_rn(r3 < NO ? W3[c3 * NO + r3] : 0.f);
            }
        }
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
        out4[c * 4 + 3] = acc * rsqrtf(1.f + r * r) / kick_coef(a, run);
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
    return sizeof(bf16) * (NH * KP1 + 2 * NH * KP2 + 8 * KP2 + NH * KP3) + sizeof(float) * (NH + NH + 8) +
           sizeof(bf16) * (NH * NI + NH * NH + 16 * NH + NI * KP2) + 640;
}

NNWeightsMut nn_carve(void *base) {
    NNWeightsMut w{};
    char *p = static_cast<char *>(base);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 15) / 16 * 16;
        return q;
    };
    w.w1t = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * KP1));
    w.w2t = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * KP2));
    w.w2n = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * KP2));
    w.w3t = reinterpret_cast<bf16 *>(take(sizeof(bf16) * 8 * KP2));
    w.w3n = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * KP3));
    w.b1 = reinterpret_cast<float *>(take(sizeof(float) * NH));
    w.b2 = reinterpret_cast<float *>(take(sizeof(float) * NH));
    w.b3 = reinterpret_cast<float *>(take(sizeof(float) * 8));
    w.w1c = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * NI));
    w.w2c = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NH * NH));
    w.w3c = reinterpret_cast<bf16 *>(take(sizeof(bf16) * 16 * NH));
    w.w1n = reinterpret_cast<bf16 *>(take(sizeof(bf16) * NI * KP2));
    return w;
}

cudaError_t launch_nn_pack(const float *theta, const NNWeightsMut &w, cudaStream_t st) {
    k_nn_pack<<<(NH * KP2 + 255) / 256, 256, 0, st>>>(theta, w);
    return cudaGetLastError();
}

template <int K1, int LB>
constexpr size_t wgrad_smem() {
    return sizeof(bf16) * TILE * ((K1 + 8) + (LB + 8));
}

cudaError_t nn_prepare() {
    cudaError_t e;
    const int fs = (int)SmemFwd::BYTES, bs = (int)SmemBwd::BYTES;
    if ((e = cudaFuncSetAttribute(k_mlp_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, bs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_wgrad<NI, NH, NH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)wgrad_smem<NI, NH>())) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_wgrad<NH, NH, NH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)wgrad_smem<NH, NH>())) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_wgrad<NH, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)wgrad_smem<NH, 8>())) != cudaSuccess)
        return e;
    return cudaSuccess;
}

namespace {
unsigned persistent_grid(int64_t tiles) {
    const int64_t cap = 2 * 152;  // two 256-thread blocks per SM (128 registers a thread)
    return (unsigned)(tiles < cap ? tiles : cap);
}
}  // namespace

cudaError_t launch_nn_fwd(const NNArgs &a, int64_t cells, bool train, cudaStream_t st) {
    const int64_t tiles = cells / TILE;
    if (train)
        k_mlp_fwd<true><<<persistent_grid(tiles), THREADS, SmemFwd::BYTES, st>>>(a, tiles);
    else
        k_mlp_fwd<false><<<persistent_grid(tiles), THREADS, SmemFwd::BYTES, st>>>(a, tiles);
    return cudaGetLastError();
}

cudaError_t launch_nn_bwd(const NNArgs &a, int64_t cells, cudaStream_t st) {
    const int64_t tiles = cells / TILE;
    k_mlp_bwd<<<persistent_grid(tiles), THREADS, SmemBwd::BYTES, st>>>(a, tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // weight gradients: dW1 = X^T g1, dW2 = h1^T g2, dW3 = h2^T g3
    const unsigned grid = persistent_grid(tiles);
    float *dW1 = a.grad, *dW2 = dW1 + NI * NH + NH, *dW3 = dW2 + NH * NH + NH;
    k_wgrad<NI, NH, NH><<<grid, THREADS, wgrad_smem<NI, NH>(), st>>>(a.xg, a.g1g, cells, dW1, NH, NH);
    k_wgrad<NH, NH, NH><<<grid, THREADS, wgrad_smem<NH, NH>(), st>>>(a.h1g, a.g2g, cells, dW2, NH, NH);
    k_wgrad<NH, 8, 8><<<grid, THREADS, wgrad_smem<NH, 8>(), st>>>(a.h2g, a.g3g, cells, dW3, NO, NO);
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
