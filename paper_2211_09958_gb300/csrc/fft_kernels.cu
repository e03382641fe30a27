// The library's own 3D real FFT for power-of-two meshes (16 <= n <= 1024),
// in three passes per direction, laid out for the PM pipeline:
//
//   real meshes     [run][x][y][z][G] floats, G = 1 (density) or 4
//                   (interleaved adjoint sources / force components)
//   spectra         [field][run][kz / 8][x][y][kz % 8] complex ("blocked":
//                   8 consecutive kz per 64-byte block), kz = 0 .. n/2 valid
//                   out of zc = n/2 + 1 rounded up to 8 (pad kept at 0)
//
//   z pass  (R2C / C2R)  rows of n reals as n/2-point complex FFTs with the
//                        even/odd packing; reads or writes the interleaved
//                        real mesh and the spectrum rows
//   pencil  (y and x)    one kz block transformed along y (a contiguous
//                        64 KB slab at n = 1024) or x (rows 64 KB apart)
//
// Conventions match cuFFT's unnormalised R2C / C2R: forward
// X_k = sum_n x_n e^{-2 pi i k n / n}, inverse without 1/n.  The spectral
// kernels apply the 1/n^3.
//
// A line of L = M1 * M2 complex points (M1 <= M2, both powers of two) is
// transformed by the four-step method: M1 threads each do an M2-point FFT in
// registers on a stride-M1 subsequence, multiply by W_L^{n1 k2}, exchange
// through shared memory (pitch M2 + 1 to spread banks), and each thread then
// does M2 / M1 of the M2 M1-point FFTs, so that no thread idles.  The
// register FFTs are radix-2 decimation in frequency (bit-reversed output),
// fully unrolled.  Twiddles come from a table of W_1024^j computed in double
// precision on the host; the 32 register-FFT twiddles sit in constant memory.

#include <cuda.h>

#include <cmath>

#include "pm_internal.h"

namespace pmgb {

__constant__ float2 c_w32[32];  // e^{-2 pi i k / 32}

namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }
__host__ __device__ constexpr int bitrev(int k, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r = (r << 1) | ((k >> i) & 1);
    return r;
}
// L = lsplit(L) * msplit(L): lsplit(L) <= msplit(L) <= 32, lsplit the number
// of threads per line.
__host__ __device__ constexpr int msplit(int l) { return 1 << ((ilog2(l) + 1) / 2); }
__host__ __device__ constexpr int lsplit(int l) { return l / msplit(l); }
__host__ __device__ constexpr int line_pitch(int l) { return l + msplit(l) + 2; }  // >= M1 (M2 + 1), even

// In-register radix-2 DIF FFT of R <= 32 points; v[i] ends as X[bitrev(i)].
template <int R, bool INV>
__device__ __forceinline__ void reg_fft(float2 (&v)[R]) {
#pragma unroll
    for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int j = 0; j < R; j += 2 * span) {
#pragma unroll
            for (int k = 0; k < span; ++k) {
                const float2 a = v[j + k], b = v[j + k + span];
                v[j + k] = cadd(a, b);
                const float2 d = csub(a, b);
                if (k == 0) {
                    v[j + k + span] = d;
                } else {
                    float2 w = c_w32[k * (32 / (2 * span))];
                    if (INV) w.y = -w.y;
                    v[j + k + span] = cmul(d, w);
                }
            }
        }
    }
}

// Steps 2-4 of the four-step FFT once thread t holds its M2 points
// v[n2] = x[t + M1 n2]: transform, twiddle, exchange through `line`
// (pitch >= M1 (M2 + 1)), then the M1-point transforms of columns
// c = t, t + M1, ...; the result X[k] lands in line[k] (natural order).
// Every lane of the warp must call it (it uses __syncwarp).
template <int L, bool INV>
__device__ __forceinline__ void line_fft_regs(float2 (&v)[msplit(L)], float2 *line, int t,
                                              const float2 *__restrict__ tw) {
    constexpr int M1 = lsplit(L), M2 = msplit(L);
    reg_fft<M2, INV>(v);
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) {
        float2 w = __ldg(tw + t * k2 * (1024 / L));
        if (INV) w.y = -w.y;
        line[t * (M2 + 1) + k2] = cmul(v[bitrev(k2, ilog2(M2))], w);
    }
    __syncwarp();
    float2 u[M2 / M1][M1];
#pragma unroll
    for (int j = 0; j < M2 / M1; ++j)
#pragma unroll
        for (int n1 = 0; n1 < M1; ++n1) u[j][n1] = line[n1 * (M2 + 1) + t + M1 * j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < M2 / M1; ++j) {
        reg_fft<M1, INV>(u[j]);
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) line[t + M1 * j + M2 * k1] = u[j][bitrev(k1, ilog2(M1))];
    }
    __syncwarp();
}

// Four-step FFT of one line of L points held in shared memory, by the M1
// threads t = 0 .. M1-1 of one warp (or sub-warp).
template <int L, bool INV>
__device__ __forceinline__ void line_fft(float2 *line, int t, const float2 *__restrict__ tw) {
    constexpr int M1 = lsplit(L), M2 = msplit(L);
    float2 v[M2];
#pragma unroll
    for (int n2 = 0; n2 < M2; ++n2) v[n2] = line[t + M1 * n2];
    __syncwarp();
    line_fft_regs<L, INV>(v, line, t, tw);
}

// --------------------------------------------------------------- z pass ---

// Z pass of n-point rows, G lines per row, about T threads per block.
template <int N, int G, int T = 256>
struct ZShape {
    static constexpr int M = N / 2, TL = lsplit(M), LP = line_pitch(M);
    static constexpr int Y = (T / TL / G) < N ? (T / TL / G) : N;  // rows per block
    static constexpr int LINES = Y * G, THREADS = LINES * TL;
};

// Forward: G interleaved real fields -> spectrum fields 0 .. G-1.  STAGE
// (G = 4, autotuned): the block's rows arrive through coalesced 16-byte
// loads into the line buffers instead of per-thread strided loads.
template <int N, int G, int T, bool STAGE>
__global__ void __launch_bounds__(T) k_fft_z_fwd(const float *__restrict__ in, float2 *spec, FftGeom fg) {
    using S = ZShape<N, G, T>;
    constexpr int M = S::M, TL = S::TL, Y = S::Y, LP = S::LP;
    extern __shared__ float4 smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int tid = threadIdx.x, line = tid / TL, t = tid % TL;
    constexpr int NYB = N / Y;
    const int y0 = (int)(blockIdx.x % NYB) * Y;
    const int64_t bx = blockIdx.x / NYB;  // run * N + x
    const int yl = line / G, g = line % G;
    if (G == 4 && STAGE) {
        // line (yl, g) gets the reals of row y0 + yl, field g, as floats
        // 0 .. N-1, from coalesced 16-byte loads (one float4 = the 4 fields
        // of one cell)
        const float4 *src = reinterpret_cast<const float4 *>(in) + (bx * N + y0) * (int64_t)N;
        float *fl = reinterpret_cast<float *>(sm);
        for (int e = tid; e < Y * N; e += S::THREADS) {
            const float4 v = __ldg(src + e);
            float *l0 = fl + (e / N) * 4 * (2 * LP) + (e % N);
            l0[0] = v.x;
            l0[2 * LP] = v.y;
            l0[4 * LP] = v.z;
            l0[6 * LP] = v.w;
        }
        __syncthreads();
        line_fft<M, false>(sm + line * LP, t, fg.tw);
    } else {
        // point n of line (row y0 + yl, field g) is the complex pair of reals
        // (2n, 2n + 1), i.e. floats G (2n) + g and G (2n + 1) + g of the row
        constexpr int M1 = lsplit(M), M2 = msplit(M);
        const float *row = in + ((bx * N + y0 + yl) * (int64_t)N) * G + g;
        float2 v[M2];
#pragma unroll
        for (int n2 = 0; n2 < M2; ++n2) {
            const int n = t + M1 * n2;
            if (G == 1)
                v[n2] = __ldg(reinterpret_cast<const float2 *>(row) + n);
            else
                v[n2] = make_float2(__ldg(row + G * 2 * n), __ldg(row + G * (2 * n + 1)));
        }
        line_fft_regs<M, false>(v, sm + line * LP, t, fg.tw);
    }
    const float2 *Lz = sm + line * LP;
    // element kz of this row sits at dst + (kz / 8) * N^2 * 8 + kz % 8
    const int64_t run = bx / N, xx = bx % N;
    float2 *dst = spec + g * fg.fstride + (run * (fg.zc / 8) * N * N + xx * N + y0 + yl) * 8;
    constexpr int64_t KB = (int64_t)N * N * 8;
    auto at = [&](int kz) -> float2 & { return dst[(kz >> 3) * KB + (kz & 7)]; };
    for (int k = t; k <= M / 2; k += TL) {
        const float2 zk = Lz[k], zm = Lz[(M - k) & (M - 1)];
        const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        const float2 WO = cmul(__ldg(fg.tw + k * (1024 / N)), O);
        at(k) = cadd(E, WO);
        const float2 r = csub(E, WO);
        if (k == 0)
            at(M) = make_float2(r.x, -r.y);
        else if (k < M / 2)
            at(M - k) = make_float2(r.x, -r.y);
    }
}

// Bounded wait on an mbarrier phase (TMA completion).
__device__ __forceinline__ bool tma_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); ++it) {
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

// Inverse: spectrum fields 0 .. GS-1 -> real mesh with GO interleaved
// slots per cell (GO = 4: slots >= GS written as 0; GO = 1: plain rows), or
// for GO = 2 two planar meshes, field 1 nb n^3 floats after field 0.
// TMA: the block's Y rows of each field, kz blocks 0 .. M/8, arrive in
// shared memory by one 5-D tensor copy per field ([16 floats][y][x][kz
// block][field, run]; box 16 x Y x 1 x (M/8 + 1) x 1) instead of per-thread
// loads; the staged rows share the space of the line buffers (consumed
// into registers before the transforms write there).
template <int N, int GS, int GO, int T, bool TMA>
__global__ void __launch_bounds__(T) k_fft_z_inv(const float2 *__restrict__ spec, float *out, FftGeom fg,
                                                 const __grid_constant__ CUtensorMap tmap) {
    using S = ZShape<N, GO, T>;
    constexpr int M = S::M, TL = S::TL, Y = S::Y, LP = S::LP;
    constexpr int NB = M / 8 + 1;  // kz blocks holding kz = 0 .. M
    extern __shared__ __align__(128) float4 smraw[];  // TMA destination: 128-byte aligned
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int tid = threadIdx.x, line = tid / TL, t = tid % TL;
    constexpr int NYB = N / Y;
    const int y0 = (int)(blockIdx.x % NYB) * Y;
    const int64_t bx = blockIdx.x / NYB;
    const int yl = line / GO, g = line % GO;
    if (TMA) {
        __shared__ __align__(8) uint64_t bar_mem;
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_mem);
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        int ok = 1;
        if (tid == 0) {
            constexpr uint32_t bytes = GS * NB * Y * 64;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
            const int run = (int)(bx / N), xx = (int)(bx % N);
            const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(sm);
#pragma unroll
            for (int f = 0; f < GS; ++f) {
                const int c4 = f * fg.nb + run;
                asm volatile(
                    "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst0 + f * NB * Y * 64),
                    "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(y0), "r"(xx), "r"(0), "r"(c4), "r"(bar)
                    : "memory");
            }
            ok = tma_wait(bar, 0);
            if (!ok) {
                atomicExch(fg.err, 1);
                tma_wait(bar, 0);  // let the copies in flight land before the block exits (bounded)
            }
        }
        if (!__syncthreads_and(ok)) return;
    }
    {
        // step 1 of the inverse M-point FFT starts from Z_k, k = t + M1 n2,
        // built from the half-spectrum pair (X_k, X_{M-k}):
        //   Z_k = (X_k + conj X_{M-k}) + i (X_k - conj X_{M-k}) W_N^{-k}
        // (imaginary parts of X_0 and X_M taken as zero)
        constexpr int M1 = lsplit(M), M2 = msplit(M);
        float2 v[M2];
        if (g < GS) {
            const int64_t run = bx / N, xx = bx % N;
            const float2 *src = spec + g * fg.fstride + (run * (fg.zc / 8) * N * N + xx * N + y0 + yl) * 8;
            constexpr int64_t KB = (int64_t)N * N * 8;
            // staged: field g, kz block b, row yl at sm[((g NB + b) Y + yl) 8]
            const float2 *stg = sm + ((int64_t)g * NB * Y + yl) * 8;
#pragma unroll
            for (int n2 = 0; n2 < M2; ++n2) {
                const int k = t + M1 * n2, km = M - k;
                float2 xk, xm;
                if (TMA) {
                    xk = stg[(k >> 3) * Y * 8 + (k & 7)];
                    xm = stg[(km >> 3) * Y * 8 + (km & 7)];
                } else {
                    xk = __ldg(src + (k >> 3) * KB + (k & 7));
                    xm = __ldg(src + (km >> 3) * KB + (km & 7));
                }
                if (k == 0) {
                    xk.y = 0.f;
                    xm.y = 0.f;
                }
                const float2 wf = __ldg(fg.tw + k * (1024 / N));
                const float2 A = make_float2(xk.x + xm.x, xk.y - xm.y);
                const float2 Dw = cmul(make_float2(xk.x - xm.x, xk.y + xm.y), make_float2(wf.x, -wf.y));
                v[n2] = make_float2(A.x - Dw.y, A.y + Dw.x);
            }
        } else {
#pragma unroll
            for (int n2 = 0; n2 < M2; ++n2) v[n2] = make_float2(0.f, 0.f);
        }
        if (TMA) __syncthreads();  // every staged value is in registers before the line buffers reuse the space
        line_fft_regs<M, true>(v, sm + line * LP, t, fg.tw);
    }
    __syncthreads();
    float4 *dst = reinterpret_cast<float4 *>(out + (bx * N + y0) * (int64_t)N * GO);
    if (GO == 2) {  // two planar meshes [field][run][n^3], rows of float4
        float4 *p0 = reinterpret_cast<float4 *>(out + (bx * N + y0) * (int64_t)N);
        float4 *p1 = p0 + (int64_t)fg.nb * N * N * N / 4;
        for (int e = tid; e < Y * N / 4; e += S::THREADS) {
            const int y2 = (4 * e) / N, z = (4 * e) % N;
            const float *l0 = reinterpret_cast<const float *>(sm + y2 * 2 * LP) + z;
            p0[e] = *reinterpret_cast<const float4 *>(l0);
            p1[e] = *reinterpret_cast<const float4 *>(l0 + 2 * LP);
        }
    } else if (GO == 4) {
        for (int e = tid; e < Y * N; e += S::THREADS) {
            const int y2 = e / N, z = e % N;
            const float *l0 = reinterpret_cast<const float *>(sm + y2 * 4 * LP);
            dst[e] = make_float4(l0[z], l0[2 * LP + z], l0[4 * LP + z], GS == 4 ? l0[6 * LP + z] : 0.f);
        }
    } else {
        for (int e = tid; e < Y * N / 4; e += S::THREADS) {
            const int y2 = (4 * e) / N, z = (4 * e) % N;
            dst[e] = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(sm + y2 * LP) + z);
        }
    }
}

// -------------------------------------------------------------- pencils ---

constexpr int kPencil = 8;

// Pencil of 8 adjacent columns (64 contiguous bytes per row), lines of L
// points along a strided axis.  Step 1: thread (n1, w) loads its M2 points of
// column w straight into registers (a warp covers 4 rows x 64 bytes per
// load), transforms them and writes the twiddled result to the exchange
// buffer [n1][k2][w] (n1 pitch M2*8 + 8 keeps half-warps on distinct banks);
// step 3: thread (r, w) transforms columns k2 = r, r + M1, ... over n1 and
// stores straight to global (M1 <= M2, so every thread has work).
// W = 16 (the x pass, autotuned): two adjacent y chunks, 128 contiguous
// bytes per row.
template <int L, int W = kPencil>
struct PencilShape {
    static constexpr int M1 = lsplit(L), M2 = msplit(L), THREADS = M1 * W, YP = M2 * W + W;
    static constexpr int SMEM = M1 * YP;  // complex elements
    static constexpr int MINB = THREADS > 256 ? 1 : 2;
};

template <int L, bool INV, int W>
__global__ void __launch_bounds__(PencilShape<L, W>::THREADS, PencilShape<L, W>::MINB)
    k_fft_pencil(float2 *data, PencilGeom pg, const float2 *__restrict__ tw) {
    using S = PencilShape<L, W>;
    constexpr int M1 = S::M1, M2 = S::M2, YP = S::YP;
    extern __shared__ float4 smraw[];
    float2 *ys = reinterpret_cast<float2 *>(smraw);
    const int tid = threadIdx.x, w = tid % W, r = tid / W;
    const int64_t p = blockIdx.x;
    const int64_t mid = p % pg.nmid, outer = p / pg.nmid;
    float2 *base = data + outer * pg.os + mid * pg.ms + w;
    const int ls = (int)pg.ls;  // offsets within one pencil fit in 32 bits (n * ls < 2^31)
    {
        const int n1 = r;
        float2 v[M2];
#pragma unroll
        for (int n2 = 0; n2 < M2; ++n2) v[n2] = base[(n1 + M1 * n2) * ls];
        reg_fft<M2, INV>(v);
#pragma unroll
        for (int k2 = 0; k2 < M2; ++k2) {
            float2 t = __ldg(tw + n1 * k2 * (1024 / L));
            if (INV) t.y = -t.y;
            ys[n1 * YP + k2 * W + w] = cmul(v[bitrev(k2, ilog2(M2))], t);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < M2 / M1; ++j) {
        const int k2 = r + M1 * j;
        float2 u[M1];
#pragma unroll
        for (int n1 = 0; n1 < M1; ++n1) u[n1] = ys[n1 * YP + k2 * W + w];
        reg_fft<M1, INV>(u);
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) base[(k2 + M2 * k1) * ls] = u[bitrev(k1, ilog2(M1))];
    }
}

template <int N, int G, int T, bool STAGE>
cudaError_t z_fwd_tt(const float *in, float2 *spec, const FftGeom &fg, cudaStream_t st) {
    using S = ZShape<N, G, T>;
    const size_t smem = sizeof(float2) * S::LINES * S::LP;
    cudaError_t e =
        cudaFuncSetAttribute(k_fft_z_fwd<N, G, T, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)fg.nb * N * (N / S::Y);
    k_fft_z_fwd<N, G, T, STAGE><<<(unsigned)blocks, S::THREADS, smem, st>>>(in, spec, fg);
    return cudaGetLastError();
}

template <int N, int G, int T>
cudaError_t z_fwd_t(const float *in, float2 *spec, const FftGeom &fg, cudaStream_t st) {
    if (G == 4 && fg.zstage) return z_fwd_tt<N, G, T, (G == 4)>(in, spec, fg, st);
    return z_fwd_tt<N, G, T, false>(in, spec, fg, st);
}

template <int N, int GS, int GO, int T, bool TMA>
cudaError_t z_inv_tt(const float2 *spec, float *out, const FftGeom &fg, const CUtensorMap &tmap, cudaStream_t st) {
    using S = ZShape<N, GO, T>;
    const size_t lines = sizeof(float2) * S::LINES * S::LP, staged = (size_t)GS * (S::M / 8 + 1) * S::Y * 64;
    const size_t smem = TMA && staged > lines ? staged : lines;
    cudaError_t e =
        cudaFuncSetAttribute(k_fft_z_inv<N, GS, GO, T, TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)fg.nb * N * (N / S::Y);
    k_fft_z_inv<N, GS, GO, T, TMA><<<(unsigned)blocks, S::THREADS, smem, st>>>(spec, out, fg, tmap);
    return cudaGetLastError();
}

// TMA staging where a map for this block shape exists (n >= 256, own
// transform; one map per output shape and block size), per-thread loads
// otherwise.
template <int N, int GS, int GO, int T>
cudaError_t z_inv_t(const float2 *spec, float *out, const FftGeom &fg, cudaStream_t st) {
    constexpr int ti = (GO == 4 ? 0 : (GO == 2 ? 3 : 6)) + (T == 128 ? 0 : (T == 256 ? 1 : 2));
    if (N >= 256 && fg.ztma && fg.tmaps && fg.tmaps[ti].valid)
        return z_inv_tt<N, GS, GO, T, (N >= 256)>(spec, out, fg, fg.tmaps[ti].map, st);
    static const CUtensorMap none{};
    return z_inv_tt<N, GS, GO, T, false>(spec, out, fg, none, st);
}

// Block-size variants (the autotuner's choice) only where rows are long
// enough for them to differ: n >= 256.
template <int N, int G>
cudaError_t z_fwd_n(const float *in, float2 *spec, const FftGeom &fg, cudaStream_t st) {
    if (N >= 256 && fg.zthreads == 128) return z_fwd_t<N, G, (N >= 256 ? 128 : 256)>(in, spec, fg, st);
    if (N >= 256 && fg.zthreads == 512) return z_fwd_t<N, G, (N >= 256 ? 512 : 256)>(in, spec, fg, st);
    return z_fwd_t<N, G, 256>(in, spec, fg, st);
}

template <int N, int GS, int GO>
cudaError_t z_inv_n(const float2 *spec, float *out, const FftGeom &fg, cudaStream_t st) {
    if (N >= 256 && fg.zthreads == 128) return z_inv_t<N, GS, GO, (N >= 256 ? 128 : 256)>(spec, out, fg, st);
    if (N >= 256 && fg.zthreads == 512) return z_inv_t<N, GS, GO, (N >= 256 ? 512 : 256)>(spec, out, fg, st);
    return z_inv_t<N, GS, GO, 256>(spec, out, fg, st);
}

template <int L, bool INV, int W>
cudaError_t pencil_w(float2 *data, const PencilGeom &pg, int64_t blocks, const float2 *tw, cudaStream_t st) {
    using S = PencilShape<L, W>;
    const size_t smem = sizeof(float2) * S::SMEM;
    cudaError_t e =
        cudaFuncSetAttribute(k_fft_pencil<L, INV, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_pencil<L, INV, W><<<(unsigned)blocks, S::THREADS, smem, st>>>(data, pg, tw);
    return cudaGetLastError();
}

template <int L, bool INV>
cudaError_t pencil_n(float2 *data, const PencilGeom &pg, int width, int64_t blocks, const float2 *tw,
                     cudaStream_t st) {
    return width == 16 ? pencil_w<L, INV, 16>(data, pg, blocks, tw, st) : pencil_w<L, INV, 8>(data, pg, blocks, tw, st);
}

template <int G>
cudaError_t z_fwd_g(const float *in, float2 *spec, const FftGeom &fg, cudaStream_t st) {
    switch (fg.n) {
        case 16: return z_fwd_n<16, G>(in, spec, fg, st);
        case 32: return z_fwd_n<32, G>(in, spec, fg, st);
        case 64: return z_fwd_n<64, G>(in, spec, fg, st);
        case 128: return z_fwd_n<128, G>(in, spec, fg, st);
        case 256: return z_fwd_n<256, G>(in, spec, fg, st);
        case 512: return z_fwd_n<512, G>(in, spec, fg, st);
        case 1024: return z_fwd_n<1024, G>(in, spec, fg, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int GS, int GO>
cudaError_t z_inv_g(const float2 *spec, float *out, const FftGeom &fg, cudaStream_t st) {
    switch (fg.n) {
        case 16: return z_inv_n<16, GS, GO>(spec, out, fg, st);
        case 32: return z_inv_n<32, GS, GO>(spec, out, fg, st);
        case 64: return z_inv_n<64, GS, GO>(spec, out, fg, st);
        case 128: return z_inv_n<128, GS, GO>(spec, out, fg, st);
        case 256: return z_inv_n<256, GS, GO>(spec, out, fg, st);
        case 512: return z_inv_n<512, GS, GO>(spec, out, fg, st);
        case 1024: return z_inv_n<1024, GS, GO>(spec, out, fg, st);
        default: return cudaErrorInvalidValue;
    }
}

template <bool INV>
cudaError_t pencil_l(float2 *data, const PencilGeom &pg, int width, int n, int64_t blocks, const float2 *tw,
                     cudaStream_t st) {
    switch (n) {
        case 16: return pencil_n<16, INV>(data, pg, width, blocks, tw, st);
        case 32: return pencil_n<32, INV>(data, pg, width, blocks, tw, st);
        case 64: return pencil_n<64, INV>(data, pg, width, blocks, tw, st);
        case 128: return pencil_n<128, INV>(data, pg, width, blocks, tw, st);
        case 256: return pencil_n<256, INV>(data, pg, width, blocks, tw, st);
        case 512: return pencil_n<512, INV>(data, pg, width, blocks, tw, st);
        case 1024: return pencil_n<1024, INV>(data, pg, width, blocks, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------ fused x round trip --
//
// The x pass is the last forward transform and the first inverse one, with
// the Green's-function multiply between them, so one kernel takes each x
// pencil (8 kz columns of one y row) through all three without writing the
// spectrum back in between.  Thread (r, w) of M1 x 8 runs the forward
// four-step FFT of column w and keeps X[k] for k = k2 + M2 k1, k2 = r + M1 j,
// in registers (k1 in bit-reversed order).  An inverse transform starts from
// that state:
//   x[m1 + M1 m2] = sum_k2 e^{2 pi i k2 m2 / M2} e^{2 pi i k2 m1 / L}
//                   sum_k1 Y[k2 + M2 k1] e^{2 pi i k1 m1 / M1},
// an M1-point FFT over k1 in registers, a twiddle, one shared-memory exchange
// and an M2-point FFT over k2, stored to rows m1 + M1 m2.
//
// Multipliers (the spectral kernels' definitions, with g = pref / k^2 times
// the per-axis deconvolution factors, 0 at k = 0 and in the kz padding):
//   force    F_j = i D_j g delta.  D_y and D_z are constant along an x line,
//            so F_y = i D_y phi and F_z = i D_z phi with phi = IFFT_x(g delta):
//            two inverse transforms (phi and F_x) give the three fields.
//   adjoint  psi = -i g (D_x u_x + D_y u_y + D_z u_z) and the force from
//            delta as above.  With the 4-point difference gradient, psi takes
//            one forward transform of a line built in real space (see the
//            kernel); with the exact spectral gradient, three accumulated ones.
// Fields are read before they are overwritten (in place: force 0 -> 0, 1, 2;
// adjoint 0..3 -> 0..3).

// Forward x FFT of one pencil column: X[j][i] = X[k2 + M2 bitrev(i)], k2 = r + M1 j.
template <int L>
__device__ __forceinline__ void xr_forward_regs(float2 (&v)[msplit(L)], float2 *ys, int r, int w,
                                                float2 (&X)[msplit(L) / lsplit(L)][lsplit(L)],
                                                const float2 *__restrict__ tw) {
    constexpr int M1 = lsplit(L), M2 = msplit(L), W = kPencil, YP = M2 * W + W;
    reg_fft<M2, false>(v);
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) ys[r * YP + k2 * W + w] = cmul(v[bitrev(k2, ilog2(M2))], __ldg(tw + r * k2 * (1024 / L)));
    __syncthreads();
#pragma unroll
    for (int j = 0; j < M2 / M1; ++j) {
        const int k2 = r + M1 * j;
#pragma unroll
        for (int n1 = 0; n1 < M1; ++n1) X[j][n1] = ys[n1 * YP + k2 * W + w];
        reg_fft<M1, false>(X[j]);
    }
    __syncthreads();
}

// The same from thread (r, w)'s points x = r + M1 n2 of column w in global memory.
template <int L>
__device__ __forceinline__ void xr_forward(const float2 *src, int64_t ls, float2 *ys, int r, int w,
                                           float2 (&X)[msplit(L) / lsplit(L)][lsplit(L)],
                                           const float2 *__restrict__ tw) {
    constexpr int M1 = lsplit(L), M2 = msplit(L);
    float2 v[M2];
#pragma unroll
    for (int n2 = 0; n2 < M2; ++n2) v[n2] = src[(r + M1 * n2) * ls];
    xr_forward_regs<L>(v, ys, r, w, X, tw);
}

// Inverse x FFT of Y, Y[j][k1] = Y[k2 + M2 k1] in natural k1 order (the
// first FFT runs in place on it), to rows of dst0 (times i s0 when scaled)
// and, with TWO, also dst1 times i s1.
template <int L, bool TWO>
__device__ __forceinline__ void xr_inverse(float2 (&Y)[msplit(L) / lsplit(L)][lsplit(L)], float2 *dst0, float2 *dst1,
                                           float s0, float s1, bool scaled, int64_t ls, float2 *ys, int r, int w,
                                           const float2 *__restrict__ tw) {
    constexpr int M1 = lsplit(L), M2 = msplit(L), W = kPencil, YP = M2 * W + W;
#pragma unroll
    for (int j = 0; j < M2 / M1; ++j) {
        const int k2 = r + M1 * j;
        reg_fft<M1, true>(Y[j]);
#pragma unroll
        for (int m1 = 0; m1 < M1; ++m1) {
            float2 t = __ldg(tw + k2 * m1 * (1024 / L));
            t.y = -t.y;
            ys[m1 * YP + k2 * W + w] = cmul(Y[j][bitrev(m1, ilog2(M1))], t);
        }
    }
    __syncthreads();
    float2 g[M2];
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) g[k2] = ys[r * YP + k2 * W + w];
    reg_fft<M2, true>(g);
#pragma unroll
    for (int m2 = 0; m2 < M2; ++m2) {
        const float2 x = g[bitrev(m2, ilog2(M2))];
        const int64_t off = (r + M1 * m2) * ls;
        dst0[off] = scaled ? make_float2(-s0 * x.y, s0 * x.x) : x;
        if (TWO) dst1[off] = make_float2(-s1 * x.y, s1 * x.x);
    }
    __syncthreads();
}

// Lines of 512 and more points do not keep the forward result: the force's
// second inverse transform re-runs the forward one from the input pencil
// (just read, so from L2), which halves the registers and lets two blocks
// share an SM.  With the 4-point difference gradient (FD) the adjoint builds
// psi from one forward transform (below) and takes the same form; with the
// exact spectral gradient it accumulates over three forward transforms and
// keeps one block per SM.
template <int L, bool ADJ, bool FD>
struct XRoundShape {
    static constexpr bool RELOAD = L >= 512 && (!ADJ || FD);
    static constexpr int MINB = RELOAD ? 2 : 1;
};

template <int L, bool ADJ, bool FD>
__global__ void __launch_bounds__(lsplit(L) * kPencil, XRoundShape<L, ADJ, FD>::MINB)
    k_fft_xround(float2 *spec, FftGeom fg, XRoundArgs xa) {
    constexpr int M1 = lsplit(L), M2 = msplit(L), W = kPencil, J = M2 / M1;
    extern __shared__ float4 smraw[];
    float2 *ys = reinterpret_cast<float2 *>(smraw);
    const int tid = threadIdx.x, w = tid % W, r = tid / W;
    const int kzblocks = fg.zc / W;
    const int64_t p = blockIdx.x;
    const int y = (int)(p % L);
    const int64_t outer = p / L;  // run * (zc / 8) + kz block
    const int run = (int)(outer / kzblocks);
    const int iz = (int)(outer % kzblocks) * W + w;
    const int64_t ls = (int64_t)L * W;
    float2 *base = spec + outer * ((int64_t)L * L * W) + (int64_t)y * W + w;
    const int64_t fs = fg.fstride;
    const float kyz2 = xa.kf * xa.kf * (float)((y < L / 2 ? y : y - L) * (y < L / 2 ? y : y - L) + iz * iz);
    const float dyz = iz > L / 2 ? 0.f : __ldg(xa.pref + run) * __ldg(xa.dec + y) * __ldg(xa.dec + iz);
    const float gy = __ldg(xa.grad + y), gz = iz > L / 2 ? 0.f : __ldg(xa.grad + iz);
    // g of mode k2 + M2 k1 (k2 = r + M1 j) and D_x there
    auto gmode = [&](int j, int k1, float &gx) -> float {
        const int ix = r + M1 * j + M2 * k1;
        const int nx = ix < L / 2 ? ix : ix - L;
        const float k2 = xa.kf * xa.kf * (float)(nx * nx) + kyz2;
        gx = __ldg(xa.grad + ix);
        return k2 > 0.f ? dyz * __ldg(xa.dec + ix) / k2 : 0.f;
    };
    // X[j][i] holds mode k1 = bitrev(i); Y[j][k1] is built in natural order
    float2 X[J][M1], Y[J][M1];
    if (ADJ && FD) {
        // psi = -i g sum_j D_j u_j = -g FFT_x(S_x u_x + i (D_y u_y + D_z u_z)): S_x is the periodic
        // 4-point difference along the line, whose Fourier symbol is i D_x, and D_y, D_z are
        // constant along it, so one forward transform of a line built in real space does it.
        // u_x (field 1) is staged in shared memory as [x][column] for the stencil.
#pragma unroll
        for (int n2 = 0; n2 < M2; ++n2) {
            const int x = r + M1 * n2;
            ys[x * W + w] = base[fs + x * ls];
        }
        __syncthreads();
        float2 v[M2];
#pragma unroll
        for (int n2 = 0; n2 < M2; ++n2) {
            const int x = r + M1 * n2;
            const float2 a1 = ys[((x + 1) & (L - 1)) * W + w], b1 = ys[((x - 1) & (L - 1)) * W + w];
            const float2 a2 = ys[((x + 2) & (L - 1)) * W + w], b2 = ys[((x - 2) & (L - 1)) * W + w];
            const float sx = xa.inv12h * (8.f * (a1.x - b1.x) - (a2.x - b2.x));
            const float sy = xa.inv12h * (8.f * (a1.y - b1.y) - (a2.y - b2.y));
            const float2 uy = base[2 * fs + x * ls], uz = base[3 * fs + x * ls];
            const float tx = gy * uy.x + gz * uz.x, ty = gy * uy.y + gz * uz.y;
            v[n2] = make_float2(sx - ty, sy + tx);  // S_x u_x + i t
        }
        __syncthreads();  // the stencil reads are done: the transform reuses the buffer
        xr_forward_regs<L>(v, ys, r, w, X, fg.tw);
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int k1 = 0; k1 < M1; ++k1) {
                float gx;
                const float g = gmode(j, k1, gx);
                const float2 a = X[j][bitrev(k1, ilog2(M1))];
                Y[j][k1] = make_float2(-g * a.x, -g * a.y);
            }
        xr_inverse<L, false>(Y, base + 3 * fs, nullptr, 0.f, 0.f, false, ls, ys, r, w, fg.tw);
    } else if (ADJ) {
        // psi = -i g (D_x u_x + D_y u_y + D_z u_z) from the three cotangent fields
        xr_forward<L>(base + fs, ls, ys, r, w, X, fg.tw);
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int k1 = 0; k1 < M1; ++k1) {
                float gx;
                gmode(j, k1, gx);
                const float2 u = X[j][bitrev(k1, ilog2(M1))];
                Y[j][k1] = make_float2(gx * u.x, gx * u.y);
            }
        xr_forward<L>(base + 2 * fs, ls, ys, r, w, X, fg.tw);
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int k1 = 0; k1 < M1; ++k1) {
                const float2 u = X[j][bitrev(k1, ilog2(M1))];
                Y[j][k1] = make_float2(Y[j][k1].x + gy * u.x, Y[j][k1].y + gy * u.y);
            }
        xr_forward<L>(base + 3 * fs, ls, ys, r, w, X, fg.tw);
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int k1 = 0; k1 < M1; ++k1) {
                float gx;
                const float g = gmode(j, k1, gx);
                const float2 u = X[j][bitrev(k1, ilog2(M1))];
                const float2 a = make_float2(Y[j][k1].x + gz * u.x, Y[j][k1].y + gz * u.y);
                Y[j][k1] = make_float2(g * a.y, -g * a.x);  // -i g a
            }
        xr_inverse<L, false>(Y, base + 3 * fs, nullptr, 0.f, 0.f, false, ls, ys, r, w, fg.tw);
    }
    // the force from delta (field 0): phi = IFFT_x(g delta) -> F_y, F_z; then F_x
    xr_forward<L>(base, ls, ys, r, w, X, fg.tw);
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) {
            float gx;
            const float g = gmode(j, k1, gx);
            const float2 d = X[j][bitrev(k1, ilog2(M1))];
            Y[j][k1] = make_float2(g * d.x, g * d.y);
        }
    xr_inverse<L, true>(Y, base + fs, base + 2 * fs, gy, gz, true, ls, ys, r, w, fg.tw);  // F_y, F_z
    if (XRoundShape<L, ADJ, FD>::RELOAD) xr_forward<L>(base, ls, ys, r, w, X, fg.tw);  // delta again (field 0 is intact)
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) {
            float gx;
            const float g = gmode(j, k1, gx) * gx;
            const float2 d = X[j][bitrev(k1, ilog2(M1))];
            Y[j][k1] = make_float2(-g * d.y, g * d.x);  // i D_x g delta
        }
    xr_inverse<L, false>(Y, base, nullptr, 0.f, 0.f, false, ls, ys, r, w, fg.tw);
}

// Potential form of the x round trip, for the 4-point difference gradient.
// The force F_j = i D_j g delta is S_j phi with phi = IFFT(g delta) and S_j
// the periodic 4-point difference along axis j (Fourier symbol i D_j), so a
// force evaluation needs the one inverse transform of phi, and the
// difference is taken on the real mesh afterwards (launch_grad_stencil):
//   force    field 0 (delta) -> field 0 (phi along x: g delta, inverse x)
//   adjoint  fields 0..3 (delta, u_x, u_y, u_z) -> field 0 (phi) and
//            field 1 (psi = -g FFT_x(S_x u_x + i (D_y u_y + D_z u_z)),
//            the stencil form of the fused adjoint above)
// One forward and one inverse transform in flight at a time: half the
// registers of the gradient form.
template <int L, int NF>
__global__ void __launch_bounds__(lsplit(L) * kPencil, 2)
    k_fft_xpot(float2 *spec, FftGeom fg, XRoundArgs xa, float gsign) {
    constexpr bool ADJ = NF == 4;
    constexpr int M1 = lsplit(L), M2 = msplit(L), W = kPencil, J = M2 / M1;
    extern __shared__ float4 smraw[];
    float2 *ys = reinterpret_cast<float2 *>(smraw);
    const int tid = threadIdx.x, w = tid % W, r = tid / W;
    const int kzblocks = fg.zc / W;
    const int64_t p = blockIdx.x;
    const int y = (int)(p % L);
    const int64_t outer = p / L;  // run * (zc / 8) + kz block
    const int run = (int)(outer / kzblocks);
    const int iz = (int)(outer % kzblocks) * W + w;
    const int64_t ls = (int64_t)L * W;
    float2 *base = spec + outer * ((int64_t)L * L * W) + (int64_t)y * W + w;
    const int64_t fs = fg.fstride;
    const float kyz2 = xa.kf * xa.kf * (float)((y < L / 2 ? y : y - L) * (y < L / 2 ? y : y - L) + iz * iz);
    const float dyz = iz > L / 2 ? 0.f : __ldg(xa.pref + run) * __ldg(xa.dec + y) * __ldg(xa.dec + iz);
    auto gmode = [&](int j, int k1) -> float {
        const int ix = r + M1 * j + M2 * k1;
        const int nx = ix < L / 2 ? ix : ix - L;
        const float k2 = xa.kf * xa.kf * (float)(nx * nx) + kyz2;
        return k2 > 0.f ? dyz * __ldg(xa.dec + ix) / k2 : 0.f;
    };
    float2 X[J][M1], Y[J][M1];
    if (ADJ) {
        const float gy = __ldg(xa.grad + y), gz = iz > L / 2 ? 0.f : __ldg(xa.grad + iz);
        // the line S_x u_x + i (D_y u_y + D_z u_z), u_x staged as [x][column] for the stencil
#pragma unroll
        for (int n2 = 0; n2 < M2; ++n2) {
            const int x = r + M1 * n2;
            ys[x * W + w] = base[fs + x * ls];
        }
        __syncthreads();
        float2 v[M2];
#pragma unroll
        for (int n2 = 0; n2 < M2; ++n2) {
            const int x = r + M1 * n2;
            const float2 a1 = ys[((x + 1) & (L - 1)) * W + w], b1 = ys[((x - 1) & (L - 1)) * W + w];
            const float2 a2 = ys[((x + 2) & (L - 1)) * W + w], b2 = ys[((x - 2) & (L - 1)) * W + w];
            const float sx = xa.inv12h * (8.f * (a1.x - b1.x) - (a2.x - b2.x));
            const float sy = xa.inv12h * (8.f * (a1.y - b1.y) - (a2.y - b2.y));
            const float2 uy = base[2 * fs + x * ls], uz = base[3 * fs + x * ls];
            const float tx = gy * uy.x + gz * uz.x, ty = gy * uy.y + gz * uz.y;
            v[n2] = make_float2(sx - ty, sy + tx);
        }
        __syncthreads();  // the stencil reads are done: the transform reuses the buffer
        xr_forward_regs<L>(v, ys, r, w, X, fg.tw);
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int k1 = 0; k1 < M1; ++k1) {
                const float g = gmode(j, k1);
                const float2 a = X[j][bitrev(k1, ilog2(M1))];
                Y[j][k1] = make_float2(-g * a.x, -g * a.y);
            }
        xr_inverse<L, false>(Y, base + fs, nullptr, 0.f, 0.f, false, ls, ys, r, w, fg.tw);  // psi -> field 1
    }
    xr_forward<L>(base, ls, ys, r, w, X, fg.tw);
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) {
            const float g = gsign * gmode(j, k1);
            const float2 d = X[j][bitrev(k1, ilog2(M1))];
            Y[j][k1] = make_float2(g * d.x, g * d.y);
        }
    xr_inverse<L, false>(Y, base, nullptr, 0.f, 0.f, false, ls, ys, r, w, fg.tw);  // phi -> field 0
}

template <int L, int NF>
cudaError_t xpot_l(float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st) {
    constexpr int M1 = lsplit(L), M2 = msplit(L);
    const size_t smem = sizeof(float2) * M1 * (M2 * kPencil + kPencil);  // >= L * 8 for the stencil stage
    cudaError_t e = cudaFuncSetAttribute(k_fft_xpot<L, NF == 2 ? 1 : NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)fg.nb * (fg.zc / kPencil) * L;
    if (NF == 2) {  // psi = -IFFT(g v) (field 1), then phi (field 0): two independent round trips
        k_fft_xpot<L, 1><<<(unsigned)blocks, M1 * kPencil, smem, st>>>(spec + fg.fstride, fg, xa, -1.f);
        k_fft_xpot<L, 1><<<(unsigned)blocks, M1 * kPencil, smem, st>>>(spec, fg, xa, 1.f);
    } else {
        k_fft_xpot<L, NF><<<(unsigned)blocks, M1 * kPencil, smem, st>>>(spec, fg, xa, 1.f);
    }
    return cudaGetLastError();
}

template <int NF>
cudaError_t xpot_n(float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st) {
    switch (fg.n) {
        case 16: return xpot_l<16, NF>(spec, fg, xa, st);
        case 32: return xpot_l<32, NF>(spec, fg, xa, st);
        case 64: return xpot_l<64, NF>(spec, fg, xa, st);
        case 128: return xpot_l<128, NF>(spec, fg, xa, st);
        case 256: return xpot_l<256, NF>(spec, fg, xa, st);
        case 512: return xpot_l<512, NF>(spec, fg, xa, st);
        case 1024: return xpot_l<1024, NF>(spec, fg, xa, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int L, bool ADJ, bool FD>
cudaError_t xround_l(float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st) {
    constexpr int M1 = lsplit(L), M2 = msplit(L);
    const size_t smem = sizeof(float2) * M1 * (M2 * kPencil + kPencil);  // >= L * 8 for the stencil stage
    cudaError_t e =
        cudaFuncSetAttribute(k_fft_xround<L, ADJ, FD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)fg.nb * (fg.zc / kPencil) * L;
    k_fft_xround<L, ADJ, FD><<<(unsigned)blocks, M1 * kPencil, smem, st>>>(spec, fg, xa);
    return cudaGetLastError();
}

template <int L, bool ADJ>
cudaError_t xround_fd(float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st) {
    if (ADJ && xa.fd) return xround_l<L, ADJ, ADJ>(spec, fg, xa, st);
    return xround_l<L, ADJ, false>(spec, fg, xa, st);
}

template <bool ADJ>
cudaError_t xround_n(float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st) {
    switch (fg.n) {
        case 16: return xround_fd<16, ADJ>(spec, fg, xa, st);
        case 32: return xround_fd<32, ADJ>(spec, fg, xa, st);
        case 64: return xround_fd<64, ADJ>(spec, fg, xa, st);
        case 128: return xround_fd<128, ADJ>(spec, fg, xa, st);
        case 256: return xround_fd<256, ADJ>(spec, fg, xa, st);
        case 512: return xround_fd<512, ADJ>(spec, fg, xa, st);
        case 1024: return xround_fd<1024, ADJ>(spec, fg, xa, st);
        default: return cudaErrorInvalidValue;
    }
}

// Copy between the blocked spectrum (field 0) and a plain
// [run][x][y][n/2 + 1] half spectrum.
__global__ void k_spec_copy(float2 *blocked, float2 *plain, FftGeom fg, bool to_plain) {
    const int n = fg.n, h = n / 2 + 1;
    const int64_t total = (int64_t)fg.nb * n * n * h;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(i % h);
        const int64_t row = i / h;  // (run * n + x) * n + y
        const int64_t run = row / ((int64_t)n * n), xy = row % ((int64_t)n * n);
        const int64_t b = ((run * (fg.zc / 8) + kz / 8) * n * n + xy) * 8 + kz % 8;
        if (to_plain)
            plain[i] = blocked[b];
        else
            blocked[b] = plain[i];
    }
}

}  // namespace

cudaError_t launch_spec_copy(float2 *blocked, float2 *plain, const FftGeom &fg, bool to_plain, cudaStream_t st) {
    const int64_t total = (int64_t)fg.nb * fg.n * fg.n * (fg.n / 2 + 1);
    const int64_t blocks = (total + 255) / 256;
    k_spec_copy<<<(unsigned)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, st>>>(blocked, plain, fg, to_plain);
    return cudaGetLastError();
}

bool own_fft_supported(int n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }

int own_fft_zc(int n) { return ((n / 2 + 1) + kPencil - 1) / kPencil * kPencil; }

cudaError_t upload_fft_constants(float2 *tw_dev) {
    float2 w32[32], w1024[1024];
    for (int k = 0; k < 32; ++k) w32[k] = make_float2((float)std::cos(2.0 * M_PI * k / 32), (float)-std::sin(2.0 * M_PI * k / 32));
    for (int k = 0; k < 1024; ++k)
        w1024[k] = make_float2((float)std::cos(2.0 * M_PI * k / 1024), (float)-std::sin(2.0 * M_PI * k / 1024));
    cudaError_t e = cudaMemcpyToSymbol(c_w32, w32, sizeof(w32));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(tw_dev, w1024, sizeof(w1024), cudaMemcpyHostToDevice);
}

// Rows per z-inverse block (ZShape<n, go, threads>::Y).
int z_inv_rows(int n, int threads, int go) {
    const int m = n / 2, tl = m / (1 << ((ilog2(m) + 1) / 2)), y = threads / tl / go;
    return y < n ? y : n;
}

// 5-D tensor maps over the blocked spectrum for the TMA z inverse, one per
// output shape and block size (rows per block Y): dims, innermost first,
// [16 floats][y][x][kz block][field * nb + run], box [16][Y][1][n/16 + 1][1].
// Returns false (and leaves the maps invalid) when the driver entry point is
// unavailable.
bool encode_z_inv_maps(float2 *spec, const FftGeom &fg, ZInvMap maps[Z_INV_MAPS]) {
    for (int i = 0; i < Z_INV_MAPS; ++i) maps[i].valid = false;
    if (fg.n < 256) return false;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    Encode encode = reinterpret_cast<Encode>(fn);
    const uint64_t n = fg.n;
    const cuuint64_t dims[5] = {16, n, n, (cuuint64_t)(fg.zc / 8), (cuuint64_t)(4 * fg.nb)};
    const cuuint64_t strides[4] = {64, n * 64, n * n * 64, (cuuint64_t)(fg.zc / 8) * n * n * 64};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const int threads[3] = {128, 256, 512}, go[3] = {4, 2, 1};
    bool all = true;
    for (int i = 0; i < Z_INV_MAPS; ++i) {
        const cuuint32_t box[5] = {16, (cuuint32_t)z_inv_rows(fg.n, threads[i % 3], go[i / 3]), 1,
                                   (cuuint32_t)(fg.n / 16 + 1), 1};
        const CUresult r = encode(&maps[i].map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, spec, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        maps[i].valid = r == CUDA_SUCCESS;
        all = all && maps[i].valid;
    }
    return all;
}

cudaError_t launch_fft_z_fwd(int g, const float *in, float2 *spec, const FftGeom &fg, cudaStream_t st) {
    switch (g) {
        case 4: return z_fwd_g<4>(in, spec, fg, st);
        case 2: return z_fwd_g<2>(in, spec, fg, st);
        case 1: return z_fwd_g<1>(in, spec, fg, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fft_z_inv(int gs, const float2 *spec, float *out, const FftGeom &fg, cudaStream_t st) {
    switch (gs) {
        case 4: return z_inv_g<4, 4>(spec, out, fg, st);
        case 3: return z_inv_g<3, 4>(spec, out, fg, st);
        case 2: return z_inv_g<2, 2>(spec, out, fg, st);
        case 1: return z_inv_g<1, 1>(spec, out, fg, st);
        default: return cudaErrorInvalidValue;
    }
}

// Transform fields [f0, f0 + nf) of the spectrum along y (axis 1) or x
// (axis 0), forward or inverse.  One pencil per (field, run, kz block) and
// x (y pass) or y (x pass); consecutive blocks take neighbouring pencils.
cudaError_t launch_fft_pencils(int axis, bool inverse, float2 *spec, int f0, int nf, const FftGeom &fg,
                               cudaStream_t st) {
    const int n = fg.n;
    const int width = axis == 0 && fg.xwidth == 16 ? 16 : kPencil;
    PencilGeom pg{};
    pg.nkz = 1;
    pg.nmid = n / (width / kPencil);
    pg.os = (int64_t)n * n * kPencil;
    float2 *base = spec + f0 * fg.fstride;
    if (axis == 1) {  // lines along y: a contiguous n x 8 slab
        pg.ls = kPencil;
        pg.ms = (int64_t)n * kPencil;
    } else {          // lines along x: rows n * 8 complex apart; width / 8 adjacent y per pencil
        pg.ls = (int64_t)n * kPencil;
        pg.ms = width;
    }
    const int64_t blocks = (int64_t)nf * fg.nb * (fg.zc / kPencil) * pg.nmid;
    return inverse ? pencil_l<true>(base, pg, width, n, blocks, fg.tw, st)
                   : pencil_l<false>(base, pg, width, n, blocks, fg.tw, st);
}

// Fused x round trip of the spectrum: forward x pass, spectral multiply,
// inverse x pass (force: field 0 -> fields 0..2; adjoint: fields 0..3 ->
// 0..3), replacing launch_fft_pencils(0, false, ...), the spectral kernel and
// launch_fft_pencils(0, true, ...).
cudaError_t launch_fft_xround(bool adj, float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st) {
    if (!xa.grad || !xa.dec || !xa.pref || !own_fft_supported(fg.n)) return cudaErrorInvalidValue;
    return adj ? xround_n<true>(spec, fg, xa, st) : xround_n<false>(spec, fg, xa, st);
}

// Potential form of the x round trip (k_fft_xpot): force field 0 -> 0;
// adjoint fields 0..3 -> 0 (phi), 1 (psi); adjoint with the source on the
// real mesh, fields 0, 1 -> 0 (phi), 1 (psi).  Needs the 4-point difference
// gradient (xa.fd).
cudaError_t launch_fft_xpot(int nf, float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st) {
    if (!xa.grad || !xa.dec || !xa.pref || !xa.fd || !own_fft_supported(fg.n)) return cudaErrorInvalidValue;
    switch (nf) {
        case 1: return xpot_n<1>(spec, fg, xa, st);
        case 2: return xpot_n<2>(spec, fg, xa, st);
        case 4: return xpot_n<4>(spec, fg, xa, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmgb
