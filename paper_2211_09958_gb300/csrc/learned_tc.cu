// The learned correction's network on the 5th-generation tensor cores:
// inference and the training forward (k_mlp_fwd_tc), the backward to the
// activation and feature cotangents (k_mlp_bwd_tc) and the weight gradients
// (k_wgrad_tc), for the per-cell MLP described in learned.cu (features
// asinh(rho - 1) of the 27 periodic neighbours and a; 32 -> 128 -> 128 -> 3,
// ReLU; BF16 operands, FP32 accumulation; output times 3/2 Om h added to the
// force meshes).  Each layer is one M = 128 tcgen05.mma chain whose
// accumulator lives in tensor memory.
//
// Per 128-cell tile (one row of A per cell, one TMEM lane per row):
//   features -> smem A1 (128 x 32, bf16)             all threads, gathered
//               from the feature mesh bf16(asinh(rho - 1)) (k_nn_feat)
//   D1 = A1 W1^T  (N = 128, 2 MMAs of K = 16)         one thread
//   h1 = relu(D1 + b1) -> smem A2 (128 x 128, bf16)  tcgen05.ld, all threads
//   D2 = A2 W2^T  (N = 128, 8 MMAs)
//   h2 = relu(D2 + b2) -> smem A2
//   D3 = A2 W3^T  (N = 16, rows 3..15 of W3^T zero)
// (A1 is the first 8 KB of A2: the L1 MMAs have finished reading it before
// the h1 epilogue writes there.)
//   out[cell][j] (+)= s_out (D3[j] + b3[j]), j < 3
// Training (TRAIN) also stores the features x and the activations h1, h2 as
// row-major bf16 rows [cells][32 | 128] for the backward pass.
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout
// (nn_cm_index).  A persistent block stages the weights once and runs PIPES
// independent tile pipelines of 8 warps (own A buffer, TMEM columns,
// mbarrier and named barrier), so that while one pipeline waits for its
// MMAs another runs its epilogue; two blocks share an SM (4 pipelines).
// Warp w of a pipeline reads TMEM lanes 32 (w % 4) .. + 31 (the cells of
// those rows) and columns 64 (w / 4) .. + 63 of each 128-wide accumulator;
// D1, D2 and D3 of a pipeline reuse its 128 columns in turn.
//
// Every wait on the MMA-completion mbarrier is bounded: on time-out the
// kernel sets *err, stops issuing work, frees its tensor memory and returns.

#include <cuda_bf16.h>

#include "pm_internal.h"

namespace pmgb {

namespace {

using bf16 = __nv_bfloat16;

constexpr int M = 128;          // cells per tile = TMEM lanes
constexpr int PIPES = 2;        // tile pipelines per block
constexpr int PT = 256;         // threads per pipeline: 8 warps, lane quarter w % 4, column half w / 4
constexpr int THREADS = PIPES * PT;
constexpr int NI = NN_IN, NH = NN_HID, NO = NN_OUT;
constexpr int N3 = 16;          // padded width of the last layer (M = 128 needs N % 16 == 0)
constexpr uint32_t TMEM_COLS = 128 * PIPES;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

// shared-memory carve-up (bytes); every operand base is 128-byte aligned
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + NH * NI * 2;
constexpr int OFF_W3 = OFF_W2 + NH * NH * 2;
constexpr int OFF_A = OFF_W3 + N3 * NH * 2;           // PIPES x A2 (128 x 128 bf16), A1 aliased at its start
constexpr int A_BYTES = M * NH * 2;
constexpr int OFF_B = OFF_A + PIPES * A_BYTES;        // b1[128], b2[128], b3[16] (FP32)
constexpr int OFF_BAR = OFF_B + (2 * NH + N3) * 4;    // PIPES mbarriers (8 B each)
constexpr int OFF_TMEM = OFF_BAR + 8 * PIPES;         // TMEM base address slot
constexpr int SMEM_BYTES = OFF_TMEM + 8;
static_assert(OFF_W2 % 128 == 0 && OFF_W3 % 128 == 0 && OFF_A % 128 == 0 && A_BYTES % 128 == 0, "alignment");
static_assert(OFF_BAR % 8 == 0, "mbarrier alignment");
static_assert(M * NI * 2 <= A_BYTES, "A1 fits in A2");
static_assert(2 * (SMEM_BYTES + 1024) <= 228 * 1024, "two blocks per SM");

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address >> 4 (bits
// 0-13), leading byte offset >> 4 (16-29), stride byte offset >> 4 (32-45),
// descriptor version 1 (bits 46-47); base offset, LBO mode and layout 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before();
__device__ __forceinline__ void fence_after();

// Named barrier of pipeline p (ids 1..PIPES; 0 is __syncthreads).
__device__ __forceinline__ void pipe_sync(int p) {
    asm volatile("bar.sync %0, %1;" ::"r"(p + 1), "r"(PT) : "memory");
}

__device__ __forceinline__ int pipe_and(int p, int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\tsetp.ne.b32 q, %1, 0;\n\tbar.red.and.pred o, %2, %3, q;\n\t"
        "selp.b32 %0, 1, 0, o;\n\t}\n"
        : "=r"(r)
        : "r"(pred), "r"(p + 1), "r"(PT)
        : "memory");
    return r;
}

// The pipeline's thread 0 waits for the barrier phase, the pipeline learns
// the outcome at its named barrier (so every thread takes the same branch),
// then orders its tensor-memory reads after the MMAs.
__device__ __forceinline__ bool wait_all(uint32_t bar, uint32_t &phase, int tp, int p) {
    const int ok = tp == 0 ? (int)bar_wait(bar, phase) : 1;
    const bool all = pipe_and(p, ok) != 0;
    fence_after();
    phase ^= 1;
    return all;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}

// bf16x2 of (relu(lo), relu(hi)), round to nearest even (lo in the low half).
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Columns 16 HALF .. 16 HALF + 15 of one cell's feature row (offsets
// q = 9 (ox + 1) + 3 (oy + 1) + (oz + 1) < 27, then a, then zeros), written
// as two 16-byte core-matrix rows at dst and dst + M * 16.
template <int HALF>
__device__ __forceinline__ void feature_rows(const unsigned short *f, int64_t c, int n, unsigned short afeat,
                                             char *dst) {
    const int x = (int)(c / ((int64_t)n * n)), y = (int)((c / n) % n), z = (int)(c % n);
    const int xs[3] = {x == 0 ? n - 1 : x - 1, x, x == n - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? n - 1 : y - 1, y, y == n - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? n - 1 : z - 1, z, z == n - 1 ? 0 : z + 1};
#pragma unroll
    for (int chunk = 0; chunk < 2; ++chunk) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint32_t v2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = 16 * HALF + 8 * chunk + 2 * e + h;
                if (q < 27)
                    v2[h] = __ldg(f + ((int64_t)xs[q / 9] * n + ys[(q / 3) % 3]) * n + zs[q % 3]);
                else
                    v2[h] = q == 27 ? afeat : 0u;
            }
            w[e] = v2[0] | (v2[1] << 16);
        }
        // the next 8 columns are the next K-direction core matrix, M * 16 bytes on
        *reinterpret_cast<uint4 *>(dst + chunk * M * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// One K-chain of MMAs: D[128 x n] (=|+=) A[128 x k] B[n x k]^T.
__device__ __forceinline__ void mma_chain(uint32_t d_tmem, uint32_t a_base, uint32_t b_base, int k, int n) {
    const uint32_t lbo_a = (M / 8) * 128, lbo_b = (uint32_t)(n / 8) * 128;
    for (int kk = 0; kk < k / 16; ++kk)
        mma_f16(d_tmem, sdesc(a_base + 2 * kk * lbo_a, lbo_a, 128), sdesc(b_base + 2 * kk * lbo_b, lbo_b, 128),
                idesc(n), kk > 0);
}

// 64 columns [c0, c0 + 64) of a 128-wide accumulator for this thread's row:
// + bias, ReLU, bf16, into the A2 operand (row `row`, columns c0 ..).
__device__ __forceinline__ void relu_to_a2(uint32_t taddr, const float *bias, int c0, int row, char *a2) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(taddr + c0 + 32 * h, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 8 columns = one 16-byte core-matrix row
            const int c = c0 + 32 * h + 8 * q;
            uint4 u;
            u.x = pack2_relu(v[8 * q + 0] + bias[c + 0], v[8 * q + 1] + bias[c + 1]);
            u.y = pack2_relu(v[8 * q + 2] + bias[c + 2], v[8 * q + 3] + bias[c + 3]);
            u.z = pack2_relu(v[8 * q + 4] + bias[c + 4], v[8 * q + 5] + bias[c + 5]);
            u.w = pack2_relu(v[8 * q + 6] + bias[c + 6], v[8 * q + 7] + bias[c + 7]);
            *reinterpret_cast<uint4 *>(a2 + 2 * nn_cm_index(row, c, M)) = u;
        }
    }
}

// The 128 rows x COLS columns of an A operand (core-matrix layout) to the
// row-major global rows dst [128][COLS], by the PT threads of a pipeline:
// eight lanes read one 128-byte core matrix (no bank conflict) and a warp
// writes 64 contiguous bytes of each of 8 rows.
template <int COLS>
__device__ __forceinline__ void rows_out(const char *a_op, bf16 *dst, int tp) {
    constexpr int JC = COLS / 8;
    for (int e = tp; e < M * JC; e += PT) {
        const int r = ((e >> 3) / JC) * 8 + (e & 7), j = (e >> 3) % JC;
        *reinterpret_cast<uint4 *>(dst + (int64_t)r * COLS + 8 * j) =
            *reinterpret_cast<const uint4 *>(a_op + 2 * nn_cm_index(r, 8 * j, M));
    }
}

template <bool TRAIN>
__global__ void __launch_bounds__(THREADS, 2) k_mlp_fwd_tc(NNArgs a, int64_t tiles) {
    extern __shared__ __align__(1024) char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int pipe = tid / PT, tp = tid % PT;           // pipeline and thread within it
    const int quarter = warp & 3, colhalf = (warp >> 2) & 1;
    const int row = 32 * quarter + lane;                // this thread's accumulator row (cell of the tile)
    float *bias = reinterpret_cast<float *>(sm + OFF_B);
    const uint32_t bar = smem_u32(sm + OFF_BAR + 8 * pipe);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_TMEM);

    // stage weights and biases; init the barriers; allocate tensor memory
    {
        const int4 *src[3] = {reinterpret_cast<const int4 *>(a.w.w1c), reinterpret_cast<const int4 *>(a.w.w2c),
                              reinterpret_cast<const int4 *>(a.w.w3c)};
        const int off[3] = {OFF_W1, OFF_W2, OFF_W3}, n16[3] = {NH * NI / 8, NH * NH / 8, N3 * NH / 8};
        for (int m = 0; m < 3; ++m)
            for (int k = tid; k < n16[m]; k += THREADS) reinterpret_cast<int4 *>(sm + off[m])[k] = src[m][k];
        for (int k = tid; k < 2 * NH + N3; k += THREADS)
            bias[k] = k < NH ? a.w.b1[k] : (k < 2 * NH ? a.w.b2[k - NH] : (k - 2 * NH < NO ? a.w.b3[k - 2 * NH] : 0.f));
    }
    if (tp == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tcol = *tslot + 128 * pipe;                     // this pipeline's 128 columns
    const uint32_t lane_base = tcol + ((uint32_t)(32 * quarter) << 16);
    char *abuf = sm + OFF_A + pipe * A_BYTES;
    const uint32_t sA = smem_u32(abuf);
    const uint32_t sW1 = smem_u32(sm + OFF_W1), sW2 = smem_u32(sm + OFF_W2), sW3 = smem_u32(sm + OFF_W3);

    const int n = a.n;
    const int64_t n3 = (int64_t)n * n * n;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t tile = (int64_t)blockIdx.x * PIPES + pipe; tile < tiles && ok; tile += (int64_t)gridDim.x * PIPES) {
        const int64_t cell0 = tile * M;
        const int64_t run = cell0 / n3;
        // features of cell `cl` from the bf16 feature mesh: threads 0..127 of
        // the pipeline build columns 0..15 (offsets 0..15), threads 128..255
        // columns 16..31 (offsets 16..26, a, zeros)
        {
            const int cl = tp & (M - 1);
            const int64_t c = cell0 - run * n3 + cl;
            const unsigned short *f = reinterpret_cast<const unsigned short *>(a.feat) + run * n3;
            const unsigned short afeat = __bfloat16_as_ushort(__float2bfloat16_rn(a.afeat));
            if (tp < M)
                feature_rows<0>(f, c, n, afeat, abuf + 2 * nn_cm_index(cl, 0, M));
            else
                feature_rows<1>(f, c, n, afeat, abuf + 2 * nn_cm_index(cl, 16, M));
        }
        fence_async_smem();
        fence_before();
        pipe_sync(pipe);
        // layer 1 (A1 = features, 128 x 32); in training the operand rows go out
        // to the row-major activation arrays while the MMAs read them
        if (tp == 0) {
            fence_after();
            mma_chain(tcol, sA, sW1, NI, NH);
            mma_commit(bar);
        }
        if (TRAIN) rows_out<NI>(abuf, a.xg + cell0 * NI, tp);
        ok = wait_all(bar, phase, tp, pipe);
        if (!ok) break;
        relu_to_a2(lane_base, bias, 64 * colhalf, row, abuf);
        fence_async_smem();
        fence_before();
        pipe_sync(pipe);
        // layer 2
        if (tp == 0) {
            fence_after();
            mma_chain(tcol, sA, sW2, NH, NH);
            mma_commit(bar);
        }
        if (TRAIN) rows_out<NH>(abuf, a.h1g + cell0 * NH, tp);
        ok = wait_all(bar, phase, tp, pipe);
        if (!ok) break;
        relu_to_a2(lane_base, bias + NH, 64 * colhalf, row, abuf);
        fence_async_smem();
        fence_before();
        pipe_sync(pipe);
        // layer 3
        if (tp == 0) {
            fence_after();
            mma_chain(tcol, sA, sW3, NH, N3);
            mma_commit(bar);
        }
        if (TRAIN) rows_out<NH>(abuf, a.h2g + cell0 * NH, tp);
        ok = wait_all(bar, phase, tp, pipe);
        if (!ok) break;
        if (colhalf == 0) {
            float y[4];
            tmem_ld4(lane_base, y);
            const float s_out = a.pref[run] * a.s_scale;
            float *dst = a.out + (cell0 + row) * 4;
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const float v = s_out * (y[j] + bias[2 * NH + j]);
                dst[j] = a.accumulate ? dst[j] + v : v;
            }
        }
        fence_before();
        pipe_sync(pipe);  // the A buffer and the accumulator columns are free for the next tile
        fence_after();
    }
    if (!ok && tp == 0) {
        atomicExch(a.err, 1);
        bar_wait(bar, phase ^ 1);  // the phase that timed out: let its MMAs finish (bounded)
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------ backward pass ---
//
// From the output cotangent to the activation cotangents, per 128-cell tile,
// with the same pipelines, TMEM columns and bounded waits as the forward:
//   gy = bf16(c s_out u)  -> smem A (128 x 16; columns 3.. zero), g3 row
//   D = gy W3             (N = 128: B[i][o] = W3[i][o], o < 3)
//   g2 = D [h2 > 0]       -> smem A (128 x 128), g2 row
//   D = g2 W2^T           (N = 128: B[i][o] = W2[i][o])
//   g1 = D [h1 > 0]       -> smem A, g1 row
//   D = g1 W1^T           (N = 32: B[f][o] = W1[f][o]) -> g_x row (FP32), when wanted
// u is slots 1..3 of the interleaved gradient mesh and c the run's kick
// factor.  The bias gradients are column sums of g3, g2 and g1 over the
// cells: each warp sums its 32 rows of a 32-column block by a transposing
// butterfly (lane l ends with column l), kept in registers across the tiles
// and added to the global FP32 gradient once per thread at the end.
constexpr int OFF_V2 = 0;                          // W2 as [in][out], 128 x 128
constexpr int OFF_V3 = OFF_V2 + NH * NH * 2;       // W3 as [hidden][out], 128 x 16
constexpr int OFF_V1 = OFF_V3 + NH * N3 * 2;       // W1 as [feature][hidden], 32 x 128
constexpr int OFF_BA = OFF_V1 + NI * NH * 2;       // PIPES x A (128 x 128), gy aliased at its start
constexpr int OFF_BBAR = OFF_BA + PIPES * A_BYTES;
constexpr int OFF_BTMEM = OFF_BBAR + 8 * PIPES;
constexpr int BWD_SMEM = OFF_BTMEM + 8;
static_assert(OFF_V3 % 128 == 0 && OFF_V1 % 128 == 0 && OFF_BA % 128 == 0, "alignment");
static_assert(2 * (BWD_SMEM + 1024) <= 228 * 1024, "two blocks per SM");

// Column sums of a warp's 32 rows x 32 columns (v: this lane's row): lane l
// returns the sum of column l.  31 shuffles.
__device__ __forceinline__ float column_sums32(float (&v)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;  // keep columns [s, 2s) of the current block, send [0, s)
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const float send = upper ? v[j] : v[j + s];
            const float keep = upper ? v[j + s] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack2_rn(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// 64 columns [c0, c0 + 64) of this thread's accumulator row, masked by the
// stored activation row (h > 0): bf16 into the A operand; the warp's column
// sums of the FP32 masked values added to gsum[0..1] (lane l: columns c0 + l
// and c0 + 32 + l).
__device__ __forceinline__ void masked_to_a(uint32_t taddr, int c0, int row, char *a_op, const bf16 *h_row,
                                            float (&gsum)[2], int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(taddr + c0 + 32 * h, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + 32 * h + 8 * q;
            const uint4 hv = *reinterpret_cast<const uint4 *>(h_row + c);
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {  // bf16 h > 0: sign bit clear and not +0
                if ((hw[e] & 0x8000u) || !(hw[e] & 0x7fffu)) v[8 * q + 2 * e] = 0.f;
                if ((hw[e] & 0x80000000u) || !(hw[e] & 0x7fff0000u)) v[8 * q + 2 * e + 1] = 0.f;
            }
            uint4 u;
            u.x = pack2_rn(v[8 * q + 0], v[8 * q + 1]);
            u.y = pack2_rn(v[8 * q + 2], v[8 * q + 3]);
            u.z = pack2_rn(v[8 * q + 4], v[8 * q + 5]);
            u.w = pack2_rn(v[8 * q + 6], v[8 * q + 7]);
            *reinterpret_cast<uint4 *>(a_op + 2 * nn_cm_index(row, c, M)) = u;
        }
        gsum[h] += column_sums32(v, lane);
    }
}

__global__ void __launch_bounds__(THREADS, 2) k_mlp_bwd_tc(NNArgs a, int64_t tiles) {
    extern __shared__ __align__(1024) char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int pipe = tid / PT, tp = tid % PT;
    const int quarter = warp & 3, colhalf = (warp >> 2) & 1;
    const int row = 32 * quarter + lane;
    const uint32_t bar = smem_u32(sm + OFF_BBAR + 8 * pipe);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_BTMEM);
    {
        const int4 *src[3] = {reinterpret_cast<const int4 *>(a.w.w2b), reinterpret_cast<const int4 *>(a.w.w3b),
                              reinterpret_cast<const int4 *>(a.w.w1b)};
        const int off[3] = {OFF_V2, OFF_V3, OFF_V1}, n16[3] = {NH * NH / 8, NH * N3 / 8, NI * NH / 8};
        for (int m = 0; m < 3; ++m)
            for (int k = tid; k < n16[m]; k += THREADS) reinterpret_cast<int4 *>(sm + off[m])[k] = src[m][k];
    }
    if (tp == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tcol = *tslot + 128 * pipe;
    const uint32_t lane_base = tcol + ((uint32_t)(32 * quarter) << 16);
    char *abuf = sm + OFF_BA + pipe * A_BYTES;
    const uint32_t sA = smem_u32(abuf);
    const uint32_t sV2 = smem_u32(sm + OFF_V2), sV3 = smem_u32(sm + OFF_V3), sV1 = smem_u32(sm + OFF_V1);

    const int64_t n3 = (int64_t)a.n * a.n * a.n;
    float gs3[NO] = {0.f, 0.f, 0.f}, gs2[2] = {0.f, 0.f}, gs1[2] = {0.f, 0.f};
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t tile = (int64_t)blockIdx.x * PIPES + pipe; tile < tiles && ok; tile += (int64_t)gridDim.x * PIPES) {
        const int64_t cell0 = tile * M, cell = cell0 + row;
        const int64_t run = cell0 / n3;
        // the activation rows the epilogues mask with (128 bytes each), towards L1
        // while the MMAs run
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.h2g + cell * NH + 64 * colhalf));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.h1g + cell * NH + 64 * colhalf));
        if (colhalf == 0) {  // output cotangent of this thread's cell
            const float s_out = a.pref[run] * a.s_scale * nn_kick_coef(a, run);
            const float4 u = *reinterpret_cast<const float4 *>(a.gmesh + cell * 4);
            const uint32_t g01 = pack2_rn(s_out * u.y, s_out * u.z), g2 = pack2_rn(s_out * u.w, 0.f);
            const uint4 r0 = make_uint4(g01, g2, 0u, 0u);
            *reinterpret_cast<uint4 *>(abuf + 2 * nn_cm_index(row, 0, M)) = r0;
            *reinterpret_cast<uint4 *>(abuf + 2 * nn_cm_index(row, 8, M)) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(a.g3g + cell * 8) = r0;
            float gq[NO] = {__uint_as_float(g01 << 16), __uint_as_float(g01 & 0xffff0000u), __uint_as_float(g2 << 16)};
#pragma unroll
            for (int j = 0; j < NO; ++j) {
#pragma unroll
                for (int o = 16; o; o >>= 1) gq[j] += __shfl_xor_sync(0xffffffffu, gq[j], o);
                gs3[j] += gq[j];
            }
        }
        fence_async_smem();
        fence_before();
        pipe_sync(pipe);
        if (tp == 0) {
            fence_after();
            mma_chain(tcol, sA, sV3, N3, NH);
            mma_commit(bar);
        }
        ok = wait_all(bar, phase, tp, pipe);
        if (!ok) break;
        masked_to_a(lane_base, 64 * colhalf, row, abuf, a.h2g + cell * NH, gs2, lane);
        fence_async_smem();
        fence_before();
        pipe_sync(pipe);
        if (tp == 0) {
            fence_after();
            mma_chain(tcol, sA, sV2, NH, NH);
            mma_commit(bar);
        }
        rows_out<NH>(abuf, a.g2g + cell0 * NH, tp);  // g2 rows out while the MMAs read them
        ok = wait_all(bar, phase, tp, pipe);
        if (!ok) break;
        masked_to_a(lane_base, 64 * colhalf, row, abuf, a.h1g + cell * NH, gs1, lane);
        fence_async_smem();
        fence_before();
        pipe_sync(pipe);
        if (a.gx && tp == 0) {
            fence_after();
            mma_chain(tcol, sA, sV1, NH, NI);
            mma_commit(bar);
        }
        rows_out<NH>(abuf, a.g1g + cell0 * NH, tp);
        if (a.gx) {
            ok = wait_all(bar, phase, tp, pipe);
            if (!ok) break;
            float v[16];
            tmem_ld16(lane_base + 16 * colhalf, v);
            float4 *dst = reinterpret_cast<float4 *>(a.gx + cell * NI + 16 * colhalf);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        fence_before();
        pipe_sync(pipe);
        fence_after();
    }
    if (!ok && tp == 0) {
        atomicExch(a.err, 1);
        bar_wait(bar, phase ^ 1);
    }
    if (ok) {
        const int c = 64 * colhalf + lane;
        atomicAdd(a.gb2 + c, gs2[0]);
        atomicAdd(a.gb2 + c + 32, gs2[1]);
        atomicAdd(a.gb1 + c, gs1[0]);
        atomicAdd(a.gb1 + c + 32, gs1[1]);
        if (colhalf == 0 && lane == 0)
            for (int j = 0; j < NO; ++j) atomicAdd(a.gb3 + j, gs3[j]);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------ weight gradients ---
//
// dW = sum over cells of a_c (x) b_c for one layer, on the tensor cores:
// D[i][j] += sum_k A[i][k] B[j][k] with i the 128 units of the activation
// (or cotangent) side, j the N units of the other side and k the cells, one
// tcgen05.mma chain (K = 128 cells, 8 MMAs of K = 16) per chunk of 128
// cells, accumulating in TMEM across all the chunks a block takes.
//   dW2 = h1^T g2:  A = h1 [cells][128], B = g2 [cells][128], N = 128
//   dW3 = h2^T g3:  A = h2, B = g3 [cells][8] (3 valid; zero to N = 16)
//   dW1^T = g1^T x: A = g1, B = x [cells][32], N = 32; stored transposed
// The operands are used as they lie in memory: [cells][units] rows are
// MN-major for this product (units contiguous, the cells the K dimension),
// so each 16-byte piece (cell k, units 8j .. 8j + 7) is copied with a
// coalesced load straight into its MN-major core matrix: 8 cells x 8 units,
// cell rows 16 bytes apart, unit blocks 128 bytes apart (stride byte
// offset), cell blocks R / 8 * 128 bytes apart (leading byte offset); the
// instruction descriptor marks A and B MN-major.  Two operand stages, so
// that one chunk is staged while the MMAs of the previous one run.  At the
// end each thread reads its TMEM lane (unit i) and adds its columns to the
// FP32 gradient in global memory.  Waits are bounded as in k_mlp_fwd_tc.
constexpr int WG_THREADS = 256;
constexpr int WG_K = 128;  // cells per chunk

template <int N>
struct WgShape {
    static constexpr int A_BYTES = M * WG_K * 2, B_BYTES = N * WG_K * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int OFF_BAR = 2 * STAGE, OFF_TMEM = OFF_BAR + 16, SMEM = OFF_TMEM + 8;
    static constexpr uint32_t COLS = N < 32 ? 32 : N;  // TMEM allocation: a power of two >= 32
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Instruction descriptor of the weight-gradient products: kind::f16 as
// idesc(n), with A and B MN-major (bits 15 and 16).
__host__ __device__ constexpr uint32_t idesc_mn(int n) { return idesc(n) | (1u << 15) | (1u << 16); }

// 16-byte asynchronous copy from global to shared memory; src_bytes = 0
// writes zeros without reading.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// Rows [c0, c0 + 128) of src ([cells][ld] bf16) into the MN-major core
// matrices of R units (units >= ld zero), as asynchronous copies.
template <int R>
__device__ __forceinline__ void wg_copy_mn(const bf16 *__restrict__ src, int ld, int64_t c0, char *dst, int tid) {
    constexpr int JR = R / 8;
    // e = ((k / 8) JR + j) 8 + k % 8: eight lanes fill one core matrix (128
    // contiguous bytes of shared memory, no bank conflict), and a warp reads
    // 8 cell rows of 64 bytes (R >= 32)
    for (int e = tid; e < WG_K * JR; e += WG_THREADS) {
        const int k = ((e >> 3) / JR) * 8 + (e & 7), j = (e >> 3) % JR;
        const bool in = 8 * j < ld;
        cp_async16(dst + ((k >> 3) * JR + j) * 128 + (k & 7) * 16, in ? src + (c0 + k) * ld + 8 * j : src,
                   in ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__global__ void __launch_bounds__(WG_THREADS, 1)
    k_wgrad_tc(const bf16 *__restrict__ A, const bf16 *__restrict__ B, int ldb, int64_t chunks, float *out,
               int ldo, int nvalid, int transposed, int *err) {
    using S = WgShape<N>;
    extern __shared__ __align__(1024) char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar0 = smem_u32(sm + S::OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + S::OFF_TMEM);
    if (tid == 0) {
        for (int st = 0; st < 2; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * st) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(S::COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tcol = *tslot;
    uint32_t phase[2] = {0, 0};
    int issued[2] = {0, 0};
    bool ok = true;
    int64_t it = 0;
    if (blockIdx.x < chunks) {  // chunk 0's copies; each iteration issues the next chunk's before waiting
        wg_copy_mn<M>(A, M, (int64_t)blockIdx.x * WG_K, sm, tid);
        wg_copy_mn<N>(B, ldb, (int64_t)blockIdx.x * WG_K, sm + S::A_BYTES, tid);
    }
    for (int64_t ch = blockIdx.x; ch < chunks && ok; ch += gridDim.x, ++it) {
        const int st = (int)(it & 1);
        const uint32_t bar = bar0 + 8 * st;
        const int64_t nx = ch + gridDim.x;
        if (nx < chunks) {
            const int sn = st ^ 1;
            if (issued[sn]) {  // the MMAs that read the other stage (previous chunk) must be done
                const int good = tid == 0 ? (int)bar_wait(bar0 + 8 * sn, phase[sn]) : 1;
                ok = __syncthreads_and(good) != 0;
                phase[sn] ^= 1;
                issued[sn] = 0;
                if (!ok) break;
            }
            char *na = sm + sn * S::STAGE;
            wg_copy_mn<M>(A, M, nx * WG_K, na, tid);
            wg_copy_mn<N>(B, ldb, nx * WG_K, na + S::A_BYTES, tid);
            asm volatile("cp.async.wait_group 2;" ::: "memory");  // this chunk's two groups have landed
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        char *sa = sm + st * S::STAGE, *sb = sa + S::A_BYTES;
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t lbo_a = (M / 8) * 128, lbo_b = (uint32_t)(N / 8) * 128;
            const uint32_t a_base = smem_u32(sa), b_base = smem_u32(sb);
            for (int kk = 0; kk < WG_K / 16; ++kk)
                mma_f16(tcol, sdesc(a_base + 2 * kk * lbo_a, lbo_a, 128), sdesc(b_base + 2 * kk * lbo_b, lbo_b, 128),
                        idesc_mn(N), (it > 0 || kk > 0) ? 1u : 0u);
            mma_commit(bar);
        }
        issued[st] = 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the loop (early exit on a time-out)
    // drain both stages
    for (int st = 0; st < 2; ++st) {
        if (!issued[st]) continue;
        const int good = tid == 0 ? (int)bar_wait(bar0 + 8 * st, phase[st]) : 1;
        ok = (__syncthreads_and(good) != 0) && ok;
        phase[st] ^= 1;
    }
    fence_after();
    if (ok && it > 0 && warp < 4) {  // warp w reads TMEM lanes 32 w .. 32 w + 31 (units i)
        const int i = 32 * warp + lane;
        const uint32_t lane_base = tcol + ((uint32_t)(32 * warp) << 16);
        for (int c = 0; c < N; c += 32) {
            float v[32];
            if (N >= 32) {
                tmem_ld32(lane_base + c, v);
            } else {
                float v4[4];
#pragma unroll
                for (int q = 0; q < N / 4; ++q) {
                    tmem_ld4(lane_base + 4 * q, v4);
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[4 * q + r] = v4[r];
                }
            }
#pragma unroll
            for (int j = 0; j < (N < 32 ? N : 32); ++j)
                if (c + j < nvalid) atomicAdd(transposed ? out + (c + j) * ldo + i : out + i * ldo + c + j, v[j]);
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tcol), "r"(S::COLS) : "memory");
    }
}

// Feature mesh: bf16(asinh(rho - 1)) per cell, four cells a thread; rho
// every `stride`-th float (1: a plain mesh; 4: slot 0 of the adjoint's
// interleaved paint).
__global__ void k_nn_feat(const float *__restrict__ rho, int stride, uint2 *__restrict__ feat, int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = stride == 1 ? reinterpret_cast<const float4 *>(rho)[i]
                                     : make_float4(rho[16 * i], rho[16 * i + 4], rho[16 * i + 8], rho[16 * i + 12]);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(asinhf(r.x - 1.f), asinhf(r.y - 1.f));
        const __nv_bfloat162 hi = __floats2bfloat162_rn(asinhf(r.z - 1.f), asinhf(r.w - 1.f));
        feat[i] = make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
    }
}

}  // namespace

cudaError_t launch_nn_feat(const float *rho, __nv_bfloat16 *feat, int64_t cells, cudaStream_t st, int stride) {
    if (stride != 1 && stride != 4) return cudaErrorInvalidValue;
    const int64_t n4 = cells / 4, blocks = (n4 + 255) / 256;
    k_nn_feat<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(rho, stride,
                                                                              reinterpret_cast<uint2 *>(feat), n4);
    return cudaGetLastError();
}

cudaError_t nn_tc_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_mlp_fwd_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_fwd_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, BWD_SMEM)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_wgrad_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  WgShape<128>::SMEM)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_wgrad_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  WgShape<32>::SMEM)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_wgrad_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  WgShape<16>::SMEM)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

// The three weight gradients of one training step on the tensor cores,
// from the activations the training forward stored (x, h1, h2) and the
// cotangents the backward stored (g1, g2, g3); added to a.grad.
cudaError_t launch_nn_wgrad_tc(const NNArgs &a, int64_t cells, cudaStream_t st) {
    const int64_t chunks = cells / WG_K;
    // blocks per SM as shared memory allows (128, 80 and 72 KB)
    auto grid = [&](int per_sm) { return (unsigned)(chunks < 152 * per_sm ? chunks : 152 * per_sm); };
    float *dW1 = a.grad, *dW2 = dW1 + NI * NH + NH, *dW3 = dW2 + NH * NH + NH;
    k_wgrad_tc<128><<<grid(1), WG_THREADS, WgShape<128>::SMEM, st>>>(a.h1g, a.g2g, NH, chunks, dW2, NH, NH, 0, a.err);
    k_wgrad_tc<16><<<grid(3), WG_THREADS, WgShape<16>::SMEM, st>>>(a.h2g, a.g3g, 8, chunks, dW3, NO, NO, 0, a.err);
    k_wgrad_tc<32><<<grid(2), WG_THREADS, WgShape<32>::SMEM, st>>>(a.g1g, a.xg, NI, chunks, dW1, NH, NI, 1, a.err);
    return cudaGetLastError();
}

// Backward of one training step: activation cotangents, bias gradients and
// (a.gx) the feature cotangent, then the weight gradients.
cudaError_t launch_nn_bwd(const NNArgs &a, int64_t cells, cudaStream_t st) {
    const int64_t tiles = cells / M;
    const int64_t want = (tiles + PIPES - 1) / PIPES;
    const int64_t cap = 2 * 152;
    k_mlp_bwd_tc<<<(unsigned)(want < cap ? want : cap), THREADS, BWD_SMEM, st>>>(a, tiles);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_nn_wgrad_tc(a, cells, st);
}

cudaError_t launch_nn_fwd_tc(const NNArgs &a, int64_t cells, cudaStream_t st, bool train) {
    const int64_t tiles = cells / M;
    const int64_t want = (tiles + PIPES - 1) / PIPES;
    const int64_t cap = 2 * 152;  // two blocks per SM: 2 x 256 TMEM columns, 2 x ~109 KB shared memory
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    if (train)
        k_mlp_fwd_tc<true><<<grid, THREADS, SMEM_BYTES, st>>>(a, tiles);
    else
        k_mlp_fwd_tc<false><<<grid, THREADS, SMEM_BYTES, st>>>(a, tiles);
    return cudaGetLastError();
}

}  // namespace pmgb
