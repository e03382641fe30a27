// Cloud-in-cell (CIC) particle kernels: mass assignment (paint) fused with
// the drift / reverse drift that precedes it, and interpolation (read) fused
// with the kick / adjoint update that follows it.
//
// Paper (pmwd, arXiv:2211.09958), Summary: a particle-mesh simulation whose
// gradients come from the adjoint method with reverse time integration.
// CIC weights: u = x / h, i0 = floor(u), f = u - i0, per-axis weights
// (1 - f, f) at (i0, i0 + 1) mod n_m; W = product over axes; dW/dx uses the
// one-sided slopes (-1/h, +1/h).  Particle positions are rebuilt from the
// FP32 displacement and the integer lattice index, x / h = i n_m / n_p + 1/2
// + s / h, splitting off the integer cell so that precision does not depend
// on the box size.

#include "pm_internal.h"

namespace pmgb {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void lattice_ijk(int64_t i, int np, int li[3]) {
    const int64_t np2 = (int64_t)np * np;
    const int64_t ix = i / np2;
    const int64_t r = i - ix * np2;
    const int64_t iy = r / np;
    li[0] = (int)ix;
    li[1] = (int)iy;
    li[2] = (int)(r - iy * np);
}

// Cell index and fraction along one axis.
__device__ __forceinline__ void axis_cell(int li, float sv, const Geom &g, int &c, float &f) {
    int qi;
    float qf;
    if (g.ratio) {
        qi = li * g.ratio;
        qf = 0.f;
    } else {
        const int64_t num = (int64_t)li * g.nm;
        qi = (int)(num / g.np);
        qf = (float)(num - (int64_t)qi * g.np) * g.inv_np;
    }
    const float t = qf + 0.5f + sv * g.inv_h;
    const float fl = floorf(t);
    int ci = (qi + (int)fl) % g.nm;
    if (ci < 0) ci += g.nm;
    c = ci;
    f = t - fl;
}

__device__ __forceinline__ void locate(int64_t i, float sx, float sy, float sz, const Geom &g, int c[3],
                                       float f[3]) {
    int li[3];
    lattice_ijk(i, g.np, li);
    axis_cell(li[0], sx, g, c[0], f[0]);
    axis_cell(li[1], sy, g, c[1], f[1]);
    axis_cell(li[2], sz, g, c[2], f[2]);
}

// Sum v over the block and add it to *dst (one double atomic per block).
template <int N>
__device__ __forceinline__ void block_sum_to(float (&v)[N], double *dst, int stride) {
    __shared__ float part[N][kThreads / 32];
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
        for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) part[q][w] = v[q];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            float x = lane < kThreads / 32 ? part[q][lane] : 0.f;
#pragma unroll
            for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) atomicAdd(dst + q * stride, (double)x);
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_paint(PaintArgs a) {
    const int b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    float red[1] = {0.f};
    if (i < a.g.npart) {
        const int64_t gi = ((int64_t)b * a.g.npart + i) * 3;
        float sx = a.s[gi], sy = a.s[gi + 1], sz = a.s[gi + 2];
        float wv[4] = {a.g.alpha, 0.f, 0.f, 0.f};
        if (MODE == PAINT_KDK_PRE) {
            const float4 c = a.table[a.step * a.g.nb + b];
            const float px = a.p[gi] + c.x * a.f[gi];
            const float py = a.p[gi + 1] + c.x * a.f[gi + 1];
            const float pz = a.p[gi + 2] + c.x * a.f[gi + 2];
            sx += c.y * px;
            sy += c.y * py;
            sz += c.y * pz;
            a.p[gi] = px;
            a.p[gi + 1] = py;
            a.p[gi + 2] = pz;
            a.s[gi] = sx;
            a.s[gi + 1] = sy;
            a.s[gi + 2] = sz;
        }
        if (MODE == PAINT_ADJ_DRIFT) {
            const float dr = a.table[a.step * a.g.nb + b].y;
            const float px = a.p[gi], py = a.p[gi + 1], pz = a.p[gi + 2];
            const float lx = a.lam[gi], ly = a.lam[gi + 1], lz = a.lam[gi + 2];
            red[0] = lx * px + ly * py + lz * pz;
            sx -= dr * px;
            sy -= dr * py;
            sz -= dr * pz;
            a.s[gi] = sx;
            a.s[gi + 1] = sy;
            a.s[gi + 2] = sz;
            wv[1] = a.mu[gi] + dr * lx;
            wv[2] = a.mu[gi + 1] + dr * ly;
            wv[3] = a.mu[gi + 2] + dr * lz;
            a.mu[gi] = wv[1];
            a.mu[gi + 1] = wv[2];
            a.mu[gi + 2] = wv[3];
        } else if (MODE == PAINT_ADJ) {
            wv[1] = a.mu[gi];
            wv[2] = a.mu[gi + 1];
            wv[3] = a.mu[gi + 2];
        }
        int c[3];
        float f[3];
        locate(i, sx, sy, sz, a.g, c, f);
        const int nm = a.g.nm, zs = a.mesh.zs;
        const int xs[2] = {c[0], c[0] + 1 == nm ? 0 : c[0] + 1};
        const int ys[2] = {c[1], c[1] + 1 == nm ? 0 : c[1] + 1};
        const int zz[2] = {c[2], c[2] + 1 == nm ? 0 : c[2] + 1};
        const float wx[2] = {1.f - f[0], f[0]}, wy[2] = {1.f - f[1], f[1]}, wz[2] = {1.f - f[2], f[2]};
        float *base = a.mesh.ptr + (int64_t)b * a.mesh.bstride;
        constexpr int NF = (MODE == PAINT_ADJ || MODE == PAINT_ADJ_DRIFT) ? 4 : 1;
#pragma unroll
        for (int ox = 0; ox < 2; ++ox)
#pragma unroll
            for (int oy = 0; oy < 2; ++oy) {
                const int64_t row = ((int64_t)xs[ox] * nm + ys[oy]) * zs;
#pragma unroll
                for (int oz = 0; oz < 2; ++oz) {
                    const float w = wx[ox] * wy[oy] * wz[oz];
                    const int64_t idx = row + zz[oz];
#pragma unroll
                    for (int q = 0; q < NF; ++q) atomicAdd(base + q * a.mesh.fstride + idx, w * wv[q]);
                }
            }
    }
    if (MODE == PAINT_ADJ_DRIFT) block_sum_to<1>(red, a.red + (int64_t)b * a.red_bstride, 1);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_read(ReadArgs a) {
    const int b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    float red[1] = {0.f};
    if (i < a.g.npart) {
        const int64_t gi = ((int64_t)b * a.g.npart + i) * 3;
        float sx = a.s[gi], sy = a.s[gi + 1], sz = a.s[gi + 2];
        int c[3];
        float f[3];
        locate(i, sx, sy, sz, a.g, c, f);
        const int nm = a.g.nm, zs = a.mesh.zs;
        const int xs[2] = {c[0], c[0] + 1 == nm ? 0 : c[0] + 1};
        const int ys[2] = {c[1], c[1] + 1 == nm ? 0 : c[1] + 1};
        const int zz[2] = {c[2], c[2] + 1 == nm ? 0 : c[2] + 1};
        const float wx[2] = {1.f - f[0], f[0]}, wy[2] = {1.f - f[1], f[1]}, wz[2] = {1.f - f[2], f[2]};
        const float dw[2] = {-a.g.inv_h, a.g.inv_h};
        const float *m0 = a.mesh.ptr + (int64_t)b * a.mesh.bstride;
        const float *m1 = m0 + a.mesh.fstride;
        const float *m2 = m1 + a.mesh.fstride;
        const float *m3 = m2 + a.mesh.fstride;
        float mux = 0.f, muy = 0.f, muz = 0.f;
        if (MODE == READ_ADJ) {
            mux = a.mu[gi];
            muy = a.mu[gi + 1];
            muz = a.mu[gi + 2];
        }
        float F[3] = {0.f, 0.f, 0.f}, G[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int ox = 0; ox < 2; ++ox)
#pragma unroll
            for (int oy = 0; oy < 2; ++oy) {
                const int64_t row = ((int64_t)xs[ox] * nm + ys[oy]) * zs;
#pragma unroll
                for (int oz = 0; oz < 2; ++oz) {
                    const int64_t idx = row + zz[oz];
                    if (MODE == READ_GRAD) {
                        const float v = __ldg(m0 + idx);
                        G[0] += dw[ox] * wy[oy] * wz[oz] * v;
                        G[1] += wx[ox] * dw[oy] * wz[oz] * v;
                        G[2] += wx[ox] * wy[oy] * dw[oz] * v;
                    } else {
                        const float w = wx[ox] * wy[oy] * wz[oz];
                        const float fx = __ldg(m0 + idx), fy = __ldg(m1 + idx), fz = __ldg(m2 + idx);
                        F[0] += w * fx;
                        F[1] += w * fy;
                        F[2] += w * fz;
                        if (MODE == READ_ADJ) {
                            const float gv = mux * fx + muy * fy + muz * fz + a.g.alpha * __ldg(m3 + idx);
                            G[0] += dw[ox] * wy[oy] * wz[oz] * gv;
                            G[1] += wx[ox] * dw[oy] * wz[oz] * gv;
                            G[2] += wx[ox] * wy[oy] * dw[oz] * gv;
                        }
                    }
                }
            }
        if (MODE == READ_FORCE) {
            a.f[gi] = F[0];
            a.f[gi + 1] = F[1];
            a.f[gi + 2] = F[2];
        } else if (MODE == READ_GRAD) {
            a.f[gi] = a.g.alpha * G[0];
            a.f[gi + 1] = a.g.alpha * G[1];
            a.f[gi + 2] = a.g.alpha * G[2];
        } else {
            const float4 t = a.table[a.kick_step * a.g.nb + b];
            const float ck = a.kick_sel == KICK_A ? t.x : (a.kick_sel == KICK_B ? t.z : t.w);
            if (MODE == READ_KICK_DRIFT) {
                const float dr = a.table[a.drift_step * a.g.nb + b].y;
                const float px = a.p[gi] + ck * F[0];
                const float py = a.p[gi + 1] + ck * F[1];
                const float pz = a.p[gi + 2] + ck * F[2];
                a.p[gi] = px;
                a.p[gi + 1] = py;
                a.p[gi + 2] = pz;
                a.s[gi] = sx + dr * px;
                a.s[gi + 1] = sy + dr * py;
                a.s[gi + 2] = sz + dr * pz;
            } else if (MODE == READ_HALF_KICK) {
                a.p[gi] += ck * F[0];
                a.p[gi + 1] += ck * F[1];
                a.p[gi + 2] += ck * F[2];
                a.f[gi] = F[0];
                a.f[gi + 1] = F[1];
                a.f[gi + 2] = F[2];
            } else if (MODE == READ_ADJ) {
                red[0] = mux * F[0] + muy * F[1] + muz * F[2];
                a.lam[gi] += ck * G[0];
                a.lam[gi + 1] += ck * G[1];
                a.lam[gi + 2] += ck * G[2];
                a.p[gi] -= ck * F[0];
                a.p[gi + 1] -= ck * F[1];
                a.p[gi + 2] -= ck * F[2];
            }
        }
    }
    if (MODE == READ_ADJ) block_sum_to<1>(red, a.red + (int64_t)b * a.red_bstride, 1);
}

__global__ void k_fill(float *ptr, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ptr[i] = v;
}

__global__ void k_unpad(const float *src, int64_t bstride, int zs, float *dst, int n) {
    const int b = blockIdx.y;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / n;
        const int z = (int)(i - row * n);
        dst[(int64_t)b * n3 + i] = src[(int64_t)b * bstride + row * zs + z];
    }
}

__global__ void k_kick(Geom g, float *p, const float *f, const float4 *table, int step, int sel, float sign) {
    const int b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= g.npart) return;
    const float4 t = table[step * g.nb + b];
    const float c = sign * (sel == KICK_A ? t.x : (sel == KICK_B ? t.z : t.w));
    const int64_t gi = ((int64_t)b * g.npart + i) * 3;
    p[gi] += c * f[gi];
    p[gi + 1] += c * f[gi + 1];
    p[gi + 2] += c * f[gi + 2];
}

// d = (mesh - 1) - target; acc[b] += sum d^2; mesh <- 2 d / n^3 (in place).
__global__ void __launch_bounds__(kThreads) k_mse(MeshRef mesh, const float *target, int n, double *acc) {
    const int b = blockIdx.y;
    const int64_t n3 = (int64_t)n * n * n;
    const float scale = 2.f / (float)n3;
    double sum = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n3; i += (int64_t)gridDim.x * kThreads) {
        const int64_t row = i / n;
        float *m = mesh.ptr + (int64_t)b * mesh.bstride + row * mesh.zs + (i - row * n);
        const float d = (*m - 1.f) - target[(int64_t)b * n3 + i];
        sum += (double)d * d;
        *m = scale * d;
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __shared__ double part[kThreads / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += part[w];
        atomicAdd(acc + b, t);
    }
}

dim3 particle_grid(const Geom &g) { return dim3((unsigned)((g.npart + kThreads - 1) / kThreads), g.nb); }

}  // namespace

cudaError_t launch_paint(int mode, const PaintArgs &a, cudaStream_t st) {
    const dim3 grid = particle_grid(a.g);
    switch (mode) {
        case PAINT_DENSITY: k_paint<PAINT_DENSITY><<<grid, kThreads, 0, st>>>(a); break;
        case PAINT_KDK_PRE: k_paint<PAINT_KDK_PRE><<<grid, kThreads, 0, st>>>(a); break;
        case PAINT_ADJ: k_paint<PAINT_ADJ><<<grid, kThreads, 0, st>>>(a); break;
        case PAINT_ADJ_DRIFT: k_paint<PAINT_ADJ_DRIFT><<<grid, kThreads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_read(int mode, const ReadArgs &a, cudaStream_t st) {
    const dim3 grid = particle_grid(a.g);
    switch (mode) {
        case READ_FORCE: k_read<READ_FORCE><<<grid, kThreads, 0, st>>>(a); break;
        case READ_KICK_DRIFT: k_read<READ_KICK_DRIFT><<<grid, kThreads, 0, st>>>(a); break;
        case READ_HALF_KICK: k_read<READ_HALF_KICK><<<grid, kThreads, 0, st>>>(a); break;
        case READ_ADJ: k_read<READ_ADJ><<<grid, kThreads, 0, st>>>(a); break;
        case READ_GRAD: k_read<READ_GRAD><<<grid, kThreads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fill(float *ptr, int64_t n, float v, cudaStream_t st) {
    const int64_t blocks = (n + kThreads - 1) / kThreads;
    k_fill<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), kThreads, 0, st>>>(ptr, n, v);
    return cudaGetLastError();
}

cudaError_t launch_unpad(const float *src, int64_t bstride, int zs, float *dst, int n, int nb, cudaStream_t st) {
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t blocks = (n3 + kThreads - 1) / kThreads;
    k_unpad<<<dim3((unsigned)(blocks < 152 * 32 ? blocks : 152 * 32), nb), kThreads, 0, st>>>(src, bstride, zs, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_mse(MeshRef mesh, const float *target, int n, int nb, double *acc, cudaStream_t st) {
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t blocks = (n3 + kThreads - 1) / kThreads;
    k_mse<<<dim3((unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), nb), kThreads, 0, st>>>(mesh, target, n, acc);
    return cudaGetLastError();
}

cudaError_t launch_kick(const Geom &g, float *p, const float *f, const float4 *table, int step, int sel,
                        float sign, cudaStream_t st) {
    k_kick<<<particle_grid(g), kThreads, 0, st>>>(g, p, f, table, step, sel, sign);
    return cudaGetLastError();
}

}  // namespace pmgb
