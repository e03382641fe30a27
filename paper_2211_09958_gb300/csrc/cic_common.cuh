// Device helpers shared by every CIC kernel: particle position -> base cell
// and fraction, and block reductions.  Binning, paint and read all call the
// same `locate`, so a particle's base cell is bit-identical in all of them.
//
// Positions are rebuilt from the FP32 displacement and the integer lattice
// index: x / h = i n_m / n_p + 1/2 + s / h (lattice half a mesh cell off the
// nodes), with the integer part of the lattice term split off so that the
// fraction's precision does not depend on the box size.
#pragma once

#include "pm_internal.h"

namespace pmgb {
namespace cic {

__device__ __forceinline__ void lattice_ijk(int64_t i, int np, int li[3]) {
    const int64_t np2 = (int64_t)np * np;
    const int64_t ix = i / np2;
    const int64_t r = i - ix * np2;
    const int64_t iy = r / np;
    li[0] = (int)ix;
    li[1] = (int)iy;
    li[2] = (int)(r - iy * np);
}

// Cell index in [0, n_m) and fraction in [0, 1) along one axis.  NaN or
// infinite displacements still give an in-range cell.
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

// TSC along one axis: nearest node j = floor(t + 1/2) of the node
// coordinate t, d = t - j in [-1/2, 1/2); c0 = j - 1 (mod n_m), the first of
// the three nodes j - 1, j, j + 1.
__device__ __forceinline__ void axis_tsc(int li, float sv, const Geom &g, int &c0, float &d) {
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
    const float fl = floorf(t + 0.5f);
    int cj = (qi + (int)fl - 1) % g.nm;
    if (cj < 0) cj += g.nm;
    c0 = cj;
    d = t - fl;
}

// The assignment stencil of one particle: K nodes per axis (2 CIC, 3 TSC),
// their weights and d weight / dx.
template <int K>
struct Stencil {
    int n[3][K];
    float w[3][K], dw[3][K];
};

template <int K>
__device__ __forceinline__ void stencil(int64_t i, float sx, float sy, float sz, const Geom &g, Stencil<K> &st) {
    const int nm = g.nm;
    if (K == 2) {
        int c[3];
        float f[3];
        locate(i, sx, sy, sz, g, c, f);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            st.n[a][0] = c[a];
            st.n[a][K - 1] = c[a] + 1 == nm ? 0 : c[a] + 1;
            st.w[a][0] = 1.f - f[a];
            st.w[a][K - 1] = f[a];
            st.dw[a][0] = -g.inv_h;
            st.dw[a][K - 1] = g.inv_h;
        }
    } else {
        int li[3];
        lattice_ijk(i, g.np, li);
        const float sv[3] = {sx, sy, sz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int c0;
            float d;
            axis_tsc(li[a], sv[a], g, c0, d);
#pragma unroll
            for (int k = 0; k < K; ++k) st.n[a][k] = c0 + k >= nm ? c0 + k - nm : c0 + k;
            const float lo = 0.5f - d, hi = 0.5f + d;
            st.w[a][0] = 0.5f * lo * lo;
            st.w[a][1] = 0.75f - d * d;
            st.w[a][K - 1] = 0.5f * hi * hi;
            st.dw[a][0] = -lo * g.inv_h;
            st.dw[a][1] = -2.f * d * g.inv_h;
            st.dw[a][K - 1] = hi * g.inv_h;
        }
    }
}

// Sum v over a block of THREADS threads and add it to dst[q * stride]
// (one double atomic per block and value).  Every thread must call it.
template <int THREADS, int N>
__device__ __forceinline__ void block_sum_to(float (&v)[N], double *dst, int stride) {
    __shared__ float part[N][THREADS / 32];
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
            float x = lane < THREADS / 32 ? part[q][lane] : 0.f;
#pragma unroll
            for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) atomicAdd(dst + q * stride, (double)x);
        }
    }
}

}  // namespace cic

// The per-mode update after a particle's force F (and, for the adjoint, the
// position VJP G) has been interpolated.  red[0] collects mu.F (cotangent of
// the kick factor), red[1] lam.p of a fused reverse drift (cotangent of Dr).
template <int MODE>
__device__ __forceinline__ void finish_read(const ReadArgs &a, int b, int64_t gi, const float s[3], const float F[3],
                                            const float G[3], const float mu[3], float red[2]) {
    if (MODE == READ_FORCE) {
#pragma unroll
        for (int j = 0; j < 3; ++j) a.f[gi + j] = F[j];
    } else if (MODE == READ_GRAD) {
#pragma unroll
        for (int j = 0; j < 3; ++j) a.f[gi + j] = a.g.alpha * G[j];
    } else {
        const float4 t = a.table[a.kick_step * a.g.nb + b];
        const float ck = a.kick_sel == KICK_A ? t.x : (a.kick_sel == KICK_B ? t.z : t.w);
        if (MODE == READ_KICK_DRIFT) {
            const float dr = a.table[a.drift_step * a.g.nb + b].y;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float pj = a.p[gi + j] + ck * F[j];
                a.p[gi + j] = pj;
                a.s[gi + j] = s[j] + dr * pj;
            }
        } else if (MODE == READ_HALF_KICK) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                a.p[gi + j] += ck * F[j];
                a.f[gi + j] = F[j];
            }
        } else if (MODE == READ_ADJ) {
            red[0] += mu[0] * F[0] + mu[1] * F[1] + mu[2] * F[2];
            float lam[3], p[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                lam[j] = a.lam[gi + j] + ck * G[j];
                p[j] = a.p[gi + j] - ck * F[j];
            }
            if (a.drift_step >= 0) {
                // reverse drift of the previous step: s -= Dr p, mu += Dr lam
                const float dr = a.table[a.drift_step * a.g.nb + b].y;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    red[1] += lam[j] * p[j];
                    a.s[gi + j] = s[j] - dr * p[j];
                    a.mu[gi + j] = mu[j] + dr * lam[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                a.lam[gi + j] = lam[j];
                a.p[gi + j] = p[j];
            }
        }
    }
}

}  // namespace pmgb
