// Particle-mesh assignment kernels (cloud-in-cell, or triangular-shaped
// cloud with solver flag 8: stencils in cic_common.cuh), one thread per particle in lattice
// order: paint with global float atomics (a single 16-byte vector atomic per
// corner when the four adjoint fields are interleaved), read with the
// kick / adjoint update fused in, and the particle-local pre-step kernels.
//
// Paper (pmwd, arXiv:2211.09958), Summary: a particle-mesh simulation whose
// gradients come from the adjoint method with reverse time integration.
// CIC weights: u = x / h, i0 = floor(u), f = u - i0, per-axis weights
// (1 - f, f) at (i0, i0 + 1) mod n_m; W = product over axes; dW/dx uses the
// one-sided slopes (-1/h, +1/h).

#include "cic_common.cuh"

namespace pmgb {

namespace {

constexpr int kThreads = 256;
using cic::block_sum_to;
using cic::locate;

// One 16-byte vector reduction (sm_90+): adds four floats at a 16-byte
// aligned address in a single L2 atomic.
__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Lattice tile of one block of the potential read (TX x TY x 16 particles, z
// fastest; 4 x 2 x 16, 4 x 4 x 16 or 8 x 4 x 16): the mesh nodes a block's
// stencils touch form a compact region that L1 holds (one thread per
// particle in lattice order touches 36 full mesh rows per lattice row
// instead), and a warp's 16 x 2 sites reach each node offset in two
// 128-byte row segments (measured at 512^3 / 1024^3 with 128 threads: the
// adjoint read 9.5 -> 8.7 ms and the kick-drift read 6.7 -> 5.9 ms against
// 8 z sites; 32 z sites were slower again).  The paints keep lattice order: tiled, they ran no faster over
// the 100-step run and the density paint ran 2x slower on a clustered state,
// where a tile's particles meet in the same cells at once.
template <int T>
struct LatticeTile {
    static constexpr int TZ = 16, TX = T >= 512 ? 8 : 4, TY = T / (TX * TZ);
};

template <int T>
__device__ __forceinline__ bool tile_particle(int np, int64_t &i) {
    using LT = LatticeTile<T>;
    const int ntz = (np + LT::TZ - 1) / LT::TZ, nty = (np + LT::TY - 1) / LT::TY;
    const int tb = blockIdx.x;
    const int iz = (tb % ntz) * LT::TZ + threadIdx.x % LT::TZ;
    const int iy = ((tb / ntz) % nty) * LT::TY + (threadIdx.x / LT::TZ) % LT::TY;
    const int ix = (tb / (ntz * nty)) * LT::TX + threadIdx.x / (LT::TZ * LT::TY);
    i = ((int64_t)ix * np + iy) * np + iz;
    return ix < np && iy < np && iz < np;
}

template <int T>
dim3 tile_grid(const Geom &g) {
    using LT = LatticeTile<T>;
    const int64_t np = g.np;
    return dim3((unsigned)(((np + LT::TX - 1) / LT::TX) * ((np + LT::TY - 1) / LT::TY) * ((np + LT::TZ - 1) / LT::TZ)),
                g.nb);
}

template <int MODE, int T, int K>
__global__ void __launch_bounds__(T) k_paint(PaintArgs a) {
    const int b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * T + threadIdx.x;
    if (i >= a.g.npart) return;
    const int64_t gi = ((int64_t)b * a.g.npart + i) * 3;
    const float sx = a.s[gi], sy = a.s[gi + 1], sz = a.s[gi + 2];
    float wv[4] = {a.g.alpha, 0.f, 0.f, 0.f};
    if (MODE == PAINT_ADJ) {
        wv[1] = a.mu[gi];
        wv[2] = a.mu[gi + 1];
        wv[3] = a.mu[gi + 2];
    }
    cic::Stencil<K> st;
    cic::stencil<K>(i, sx, sy, sz, a.g, st);
    const int nm = a.g.nm, zs = a.mesh.zs;
    float *base = a.mesh.ptr + (int64_t)b * a.mesh.bstride;
    constexpr int NF = MODE == PAINT_ADJ ? 4 : 1;
    const bool il = NF == 4 && a.mesh.il == 4;
    // density, CIC: the two z corners are adjacent floats unless the stencil
    // wraps; when both sit in one 16-byte aligned group of four they go in a
    // single vector reduction (the other two lanes add zero)
    const int z0 = st.n[2][0];
    const bool zpair = NF == 1 && K == 2 && st.n[2][1] == z0 + 1 && (z0 & 3) != 3;
#pragma unroll
    for (int ox = 0; ox < K; ++ox)
#pragma unroll
        for (int oy = 0; oy < K; ++oy) {
            const int64_t row = ((int64_t)st.n[0][ox] * nm + st.n[1][oy]) * zs;
            if (zpair) {
                float *grp = base + row + (z0 & ~3);
                if ((reinterpret_cast<uintptr_t>(grp) & 15) == 0) {
                    const float wxy = st.w[0][ox] * st.w[1][oy] * wv[0];
                    const float lo = wxy * st.w[2][0], hi = wxy * st.w[2][1];
                    const int lane = z0 & 3;  // 0, 1 or 2: lo at lane, hi at lane + 1
                    red_add_v4(grp, lane == 0 ? lo : 0.f, lane == 1 ? lo : (lane == 0 ? hi : 0.f),
                               lane == 2 ? lo : (lane == 1 ? hi : 0.f), lane == 2 ? hi : 0.f);
                    continue;
                }
            }
#pragma unroll
            for (int oz = 0; oz < K; ++oz) {
                const float w = st.w[0][ox] * st.w[1][oy] * st.w[2][oz];
                const int64_t idx = row + st.n[2][oz];
                if (il) {
                    red_add_v4(base + 4 * idx, w * wv[0], w * wv[1], w * wv[2], w * wv[3]);
                } else {
#pragma unroll
                    for (int q = 0; q < NF; ++q) atomicAdd(base + q * a.mesh.fstride + idx, w * wv[q]);
                }
            }
        }
}

// The force at the 8 CIC corners (c0 + i, c1 + j, c2 + l), i, j, l in {0, 1},
// from the potential mesh phi by the 4-point difference along each axis,
//   F_a(c) = [8 (phi(c + e_a) - phi(c - e_a)) - (phi(c + 2 e_a) - phi(c - 2 e_a))] / (12 h).
// The 56 distinct nodes: along x the 6 nodes c0 - 2 .. c0 + 3 of each of the
// 4 (y, z) corner lines, along y and z the 4 outer nodes of each line (the
// inner two are corners, already loaded).
__device__ __forceinline__ void pot_corner_forces(const float *__restrict__ phi, int lgn, float inv12h, const int c[3],
                                                  float Fc[2][2][2][3]) {
    const int m = (1 << lgn) - 1;
    auto at = [&](int x, int y, int z) {
        return __ldg(phi + ((((int64_t)(x & m) << lgn) | (y & m)) << lgn | (z & m)));
    };
    float xl[2][2][6];  // phi(c0 - 2 + k, c1 + j, c2 + l)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int k = 0; k < 6; ++k) xl[j][l][k] = at(c[0] - 2 + k, c[1] + j, c[2] + l);
    float yo[2][2][4], zo[2][2][4];  // outer nodes k = 0, 1, 4, 5 of the y and z lines
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = q < 2 ? q : q + 2;
                yo[i][l][q] = at(c[0] + i, c[1] - 2 + k, c[2] + l);
                zo[i][l][q] = at(c[0] + i, c[1] + l, c[2] - 2 + k);
            }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                // line values at offsets -2 .. +2 around the corner, per axis
                const float *x5 = &xl[j][l][i];
                const float ym2 = j == 0 ? yo[i][l][0] : yo[i][l][1], ym1 = j == 0 ? yo[i][l][1] : xl[0][l][2 + i];
                const float yp1 = j == 0 ? xl[1][l][2 + i] : yo[i][l][2], yp2 = j == 0 ? yo[i][l][2] : yo[i][l][3];
                const float zm2 = l == 0 ? zo[i][j][0] : zo[i][j][1], zm1 = l == 0 ? zo[i][j][1] : xl[j][0][2 + i];
                const float zp1 = l == 0 ? xl[j][1][2 + i] : zo[i][j][2], zp2 = l == 0 ? zo[i][j][2] : zo[i][j][3];
                Fc[i][j][l][0] = inv12h * (8.f * (x5[3] - x5[1]) - (x5[4] - x5[0]));
                Fc[i][j][l][1] = inv12h * (8.f * (yp1 - ym1) - (yp2 - ym2));
                Fc[i][j][l][2] = inv12h * (8.f * (zp1 - zm1) - (zp2 - zm2));
            }
}

template <int MODE, bool IL, int T, int K, bool POT = false>
__global__ void __launch_bounds__(T) k_read(ReadArgs a) {
    const int b = blockIdx.y;
    int64_t i = (int64_t)blockIdx.x * T + threadIdx.x;
    bool valid = i < a.g.npart;
    if (POT) valid = tile_particle<T>(a.g.np, i);  // lattice tiles: the nodes a block's stencils touch stay in L1
    float red[2] = {0.f, 0.f};
    if (valid) {
        const int64_t gi = ((int64_t)b * a.g.npart + i) * 3;
        const float sx = a.s[gi], sy = a.s[gi + 1], sz = a.s[gi + 2];
        cic::Stencil<K> st;
        cic::stencil<K>(i, sx, sy, sz, a.g, st);
        const int nm = a.g.nm, zs = a.mesh.zs;
        const float(&wx)[K] = st.w[0], (&wy)[K] = st.w[1], (&wz)[K] = st.w[2];
        const float(&dx)[K] = st.dw[0], (&dy)[K] = st.dw[1], (&dz)[K] = st.dw[2];
        const float *m0 = a.mesh.ptr + (int64_t)b * a.mesh.bstride;
        const float *m1 = m0 + a.mesh.fstride;
        const float *m2 = m1 + a.mesh.fstride;
        const float *m3 = m2 + a.mesh.fstride;
        float mu[3] = {0.f, 0.f, 0.f};
        if (MODE == READ_ADJ) {
            mu[0] = a.mu[gi];
            mu[1] = a.mu[gi + 1];
            mu[2] = a.mu[gi + 2];
        }
        float F[3] = {0.f, 0.f, 0.f}, G[3] = {0.f, 0.f, 0.f};
        float Fc[2][2][2][3];
        const float *psi = nullptr;
        if (POT) {
            const int64_t n3 = (int64_t)1 << (3 * a.lgn);
            const int c3[3] = {st.n[0][0], st.n[1][0], st.n[2][0]};
            pot_corner_forces(a.pot + (int64_t)b * n3, a.lgn, a.inv12h, c3, Fc);
            psi = a.pot + ((int64_t)a.g.nb + b) * n3;
        }
#pragma unroll
        for (int ox = 0; ox < K; ++ox)
#pragma unroll
            for (int oy = 0; oy < K; ++oy) {
                const int64_t row = ((int64_t)st.n[0][ox] * nm + st.n[1][oy]) * zs;
#pragma unroll
                for (int oz = 0; oz < K; ++oz) {
                    const int64_t idx = row + st.n[2][oz];
                    if (MODE == READ_GRAD) {
                        const float v = __ldg(m0 + idx);
                        G[0] += dx[ox] * wy[oy] * wz[oz] * v;
                        G[1] += wx[ox] * dy[oy] * wz[oz] * v;
                        G[2] += wx[ox] * wy[oy] * dz[oz] * v;
                    } else {
                        const float w = wx[ox] * wy[oy] * wz[oz];
                        float fx, fy, fz, fp = 0.f;
                        if (POT) {
                            fx = Fc[ox & 1][oy & 1][oz & 1][0];
                            fy = Fc[ox & 1][oy & 1][oz & 1][1];
                            fz = Fc[ox & 1][oy & 1][oz & 1][2];
                            if (MODE == READ_ADJ)
                                fp = __ldg(psi + ((int64_t)st.n[0][ox] * nm + st.n[1][oy]) * nm + st.n[2][oz]);
                        } else if (IL) {
                            const float4 q = __ldg(reinterpret_cast<const float4 *>(m0) + idx);
                            fx = q.x;
                            fy = q.y;
                            fz = q.z;
                            fp = q.w;
                        } else {
                            fx = __ldg(m0 + idx);
                            fy = __ldg(m1 + idx);
                            fz = __ldg(m2 + idx);
                            if (MODE == READ_ADJ) fp = __ldg(m3 + idx);
                        }
                        F[0] += w * fx;
                        F[1] += w * fy;
                        F[2] += w * fz;
                        if (MODE == READ_ADJ) {
                            const float gv = mu[0] * fx + mu[1] * fy + mu[2] * fz + a.g.alpha * fp;
                            G[0] += dx[ox] * wy[oy] * wz[oz] * gv;
                            G[1] += wx[ox] * dy[oy] * wz[oz] * gv;
                            G[2] += wx[ox] * wy[oy] * dz[oz] * gv;
                        }
                    }
                }
            }
        float s3[3] = {sx, sy, sz};
        finish_read<MODE>(a, b, gi, s3, F, G, mu, red);
    }
    if (a.zero) {  // streaming stores of zeros into the next paint's mesh, grid-strided over the run
        const int64_t stride = (int64_t)gridDim.x * T;
        float4 *z = a.zero + (int64_t)b * a.zero4;
        for (int64_t j = (int64_t)blockIdx.x * T + threadIdx.x; j < a.zero4; j += stride)
            z[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (MODE == READ_ADJ) block_sum_to<T, 2>(red, a.red + (int64_t)b * a.red_bstride, a.red2_offset);
}

// p += K_a f; s += Dr p (the pre-force half of a KDK step), or the reverse
// drift s -= Dr p with mu += Dr lam and the reduction lam . p (the cotangent
// of Dr) that opens a reverse-time adjoint step.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_pre(PreArgs a) {
    const int b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    float red[1] = {0.f};
    if (i < a.g.npart) {
        const int64_t gi = ((int64_t)b * a.g.npart + i) * 3;
        const float4 t = a.table[a.step * a.g.nb + b];
        if (MODE == PRE_KICK_DRIFT) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float pj = a.p[gi + j] + t.x * a.f[gi + j];
                a.p[gi + j] = pj;
                a.s[gi + j] += t.y * pj;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float pj = a.p[gi + j], lj = a.lam[gi + j];
                red[0] += lj * pj;
                a.s[gi + j] -= t.y * pj;
                a.mu[gi + j] += t.y * lj;
            }
        }
    }
    if (MODE == PRE_REV_DRIFT) block_sum_to<kThreads, 1>(red, a.red + (int64_t)b * a.red_bstride, 1);
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

dim3 particle_grid(const Geom &g, int t = kThreads) { return dim3((unsigned)((g.npart + t - 1) / t), g.nb); }

template <int T, int K = 2>
void paint_t(int mode, const PaintArgs &a, cudaStream_t st) {
    const dim3 grid = particle_grid(a.g, T);
    if (mode == PAINT_DENSITY)
        k_paint<PAINT_DENSITY, T, K><<<grid, T, 0, st>>>(a);
    else
        k_paint<PAINT_ADJ, T, K><<<grid, T, 0, st>>>(a);
}

template <bool IL, int T, int K>
void read_il(int mode, const ReadArgs &a, cudaStream_t st) {
    const dim3 grid = particle_grid(a.g, T);
    switch (mode) {
        case READ_FORCE: k_read<READ_FORCE, IL, T, K><<<grid, T, 0, st>>>(a); break;
        case READ_KICK_DRIFT: k_read<READ_KICK_DRIFT, IL, T, K><<<grid, T, 0, st>>>(a); break;
        case READ_HALF_KICK: k_read<READ_HALF_KICK, IL, T, K><<<grid, T, 0, st>>>(a); break;
        case READ_ADJ: k_read<READ_ADJ, IL, T, K><<<grid, T, 0, st>>>(a); break;
        default: break;
    }
}

template <int T>
void read_pot(int mode, const ReadArgs &a, cudaStream_t st) {
    const dim3 grid = tile_grid<T>(a.g);
    switch (mode) {
        case READ_FORCE: k_read<READ_FORCE, false, T, 2, true><<<grid, T, 0, st>>>(a); break;
        case READ_KICK_DRIFT: k_read<READ_KICK_DRIFT, false, T, 2, true><<<grid, T, 0, st>>>(a); break;
        case READ_HALF_KICK: k_read<READ_HALF_KICK, false, T, 2, true><<<grid, T, 0, st>>>(a); break;
        case READ_ADJ: k_read<READ_ADJ, false, T, 2, true><<<grid, T, 0, st>>>(a); break;
        default: break;
    }
}

template <int T, int K = 2>
void read_t(int mode, const ReadArgs &a, cudaStream_t st) {
    if (K == 2 && a.pot)
        read_pot<T>(mode, a, st);
    else if (a.mesh.il == 4)
        read_il<true, T, K>(mode, a, st);
    else
        read_il<false, T, K>(mode, a, st);
}

}  // namespace

cudaError_t launch_paint(int mode, const PaintArgs &a, cudaStream_t st) {
    if (mode != PAINT_DENSITY && mode != PAINT_ADJ) return cudaErrorInvalidValue;
    if (a.g.order == 3) {  // TSC: one block size
        paint_t<kThreads, 3>(mode, a, st);
        return cudaGetLastError();
    }
    switch (a.threads) {
        case 128: paint_t<128>(mode, a, st); break;
        case 512: paint_t<512>(mode, a, st); break;
        default: paint_t<256>(mode, a, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_read(int mode, const ReadArgs &a, cudaStream_t st) {
    if (mode == READ_GRAD) {
        if (a.g.order == 3)
            k_read<READ_GRAD, false, kThreads, 3><<<particle_grid(a.g), kThreads, 0, st>>>(a);
        else
            k_read<READ_GRAD, false, kThreads, 2><<<particle_grid(a.g), kThreads, 0, st>>>(a);
    } else if (mode >= READ_FORCE && mode <= READ_ADJ && a.g.order == 3) {
        if (a.pot) return cudaErrorInvalidValue;  // the potential read is CIC only
        read_t<kThreads, 3>(mode, a, st);
    } else if (mode >= READ_FORCE && mode <= READ_ADJ) {
        switch (a.threads) {
            case 128: read_t<128>(mode, a, st); break;
            case 512: read_t<512>(mode, a, st); break;
            default: read_t<256>(mode, a, st); break;
        }
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pre(int mode, const PreArgs &a, cudaStream_t st) {
    const dim3 grid = particle_grid(a.g);
    if (mode == PRE_KICK_DRIFT)
        k_pre<PRE_KICK_DRIFT><<<grid, kThreads, 0, st>>>(a);
    else
        k_pre<PRE_REV_DRIFT><<<grid, kThreads, 0, st>>>(a);
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
