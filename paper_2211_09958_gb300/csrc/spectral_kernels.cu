// Fourier-space kernels: Green's function times gradient (forward and
// adjoint), the binned power spectrum, white noise and the 2LPT spectral
// steps with their adjoints.
//
// Paper (pmwd, arXiv:2211.09958): PM gravity (Summary), power spectrum as a
// summary statistic and initial conditions as inference variables
// (Statement of Need).  The rfft grid of an n^3 real field has n x n x
// (n/2 + 1) complex entries; wavenumber index j maps to n_j = j for
// j < n/2 and j - n otherwise (the Nyquist index n/2 maps to -n/2 on the
// full axes and +n/2 on the half axis).
//   force    F_j(k) = i D_j (3/2) Om delta(k) / k^2 / n^3 (times the per-axis
//            CIC deconvolution factors, 1 unless that solver flag is set),
//            zero at k = 0;
//            D_j = (8 sin(k_j h) - sin(2 k_j h)) / (6 h), the 4-point central
//            difference gradient, from a per-axis table that is exactly zero
//            at the Nyquist index (inverse transforms real)
//   adjoint  psi(k) = sum_j conj(i D_j (3/2) Om / k^2 / n^3) u_j(k)
//   2LPT     s1_j = i k_j / k^2 delta_L, phi_ij = k_i k_j / k^2 delta_L,
//            s2_j = -i k_j / k^2 S, delta_L = noise(k) sqrt(P(k) / V_c)

#include "pm_internal.h"

namespace pmgb {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void mode_ijk(int64_t m, int n, int zc, int blk, int &ix, int &iy, int &iz) {
    if (blk) {  // [kz/8][x][y][kz%8]
        const int j = (int)(m & 7);
        int64_t r = m >> 3;
        iy = (int)(r % n);
        r /= n;
        ix = (int)(r % n);
        iz = (int)(r / n) * 8 + j;
        return;
    }
    const int64_t r = m / zc;
    iz = (int)(m - r * zc);
    const int64_t x = r / n;
    iy = (int)(r - x * n);
    ix = (int)x;
}

__device__ __forceinline__ int signed_index(int j, int n) { return j < n / 2 ? j : j - n; }

__device__ __forceinline__ float2 times_i(float2 v, float s) { return make_float2(-s * v.y, s * v.x); }

template <int T>
__global__ void __launch_bounds__(T) k_spec_force(Spec sp, const float *pref) {
    const int b = blockIdx.y;
    const int n = sp.n;
    const int64_t nmodes = (int64_t)n * n * sp.zc;
    const int64_t m = (int64_t)blockIdx.x * T + threadIdx.x;
    if (m >= nmodes) return;
    int ix, iy, iz;
    mode_ijk(m, n, sp.zc, sp.blk, ix, iy, iz);
    if (iz > n / 2) return;
    const float kx = sp.kf * signed_index(ix, n), ky = sp.kf * signed_index(iy, n), kz = sp.kf * iz;
    const float k2 = kx * kx + ky * ky + kz * kz;
    const float g = k2 > 0.f ? pref[b] / k2 * (__ldg(sp.dec + ix) * __ldg(sp.dec + iy) * __ldg(sp.dec + iz)) : 0.f;
    float2 *c0 = sp.c + (int64_t)b * sp.bstride + m;
    const float2 d = *c0;
    c0[0] = times_i(d, __ldg(sp.grad + ix) * g);
    c0[sp.fstride] = times_i(d, __ldg(sp.grad + iy) * g);
    c0[2 * sp.fstride] = times_i(d, __ldg(sp.grad + iz) * g);
}

template <int T>
__global__ void __launch_bounds__(T) k_spec_adj(Spec sp, const float *pref) {
    const int b = blockIdx.y;
    const int n = sp.n;
    const int64_t nmodes = (int64_t)n * n * sp.zc;
    const int64_t m = (int64_t)blockIdx.x * T + threadIdx.x;
    if (m >= nmodes) return;
    int ix, iy, iz;
    mode_ijk(m, n, sp.zc, sp.blk, ix, iy, iz);
    if (iz > n / 2) return;
    const float kx = sp.kf * signed_index(ix, n), ky = sp.kf * signed_index(iy, n), kz = sp.kf * iz;
    const float k2 = kx * kx + ky * ky + kz * kz;
    const float g = k2 > 0.f ? pref[b] / k2 * (__ldg(sp.dec + ix) * __ldg(sp.dec + iy) * __ldg(sp.dec + iz)) : 0.f;
    float2 *c0 = sp.c + (int64_t)b * sp.bstride + m;
    const int64_t fs = sp.fstride;
    const float2 d = c0[0], ux = c0[fs], uy = c0[2 * fs], uz = c0[3 * fs];
    const float ax = __ldg(sp.grad + ix) * g, ay = __ldg(sp.grad + iy) * g, az = __ldg(sp.grad + iz) * g;
    c0[0] = times_i(d, ax);
    c0[fs] = times_i(d, ay);
    c0[2 * fs] = times_i(d, az);
    const float2 px = times_i(ux, -ax), py = times_i(uy, -ay), pz = times_i(uz, -az);
    c0[3 * fs] = make_float2(px.x + py.x + pz.x, px.y + py.y + pz.y);
}

// |delta_k|^2 binned in |k| shells; acc[b][bin][0..2] += (n_modes, sum |k| / k_F, sum |delta|^2).
__global__ void __launch_bounds__(kThreads) k_power_bins(Spec sp, double *acc, int nbins) {
    extern __shared__ double sh[];
    const int b = blockIdx.y;
    const int n = sp.n;
    for (int q = threadIdx.x; q < 3 * nbins; q += blockDim.x) sh[q] = 0.0;
    __syncthreads();
    const int64_t nmodes = (int64_t)n * n * sp.zc;
    const float2 *c0 = sp.c + (int64_t)b * sp.bstride;
    for (int64_t m = (int64_t)blockIdx.x * kThreads + threadIdx.x; m < nmodes; m += (int64_t)gridDim.x * kThreads) {
        int ix, iy, iz;
        mode_ijk(m, n, sp.zc, sp.blk, ix, iy, iz);
        if (iz > n / 2) continue;
        const int nx = signed_index(ix, n), ny = signed_index(iy, n);
        const int64_t n2 = (int64_t)nx * nx + (int64_t)ny * ny + (int64_t)iz * iz;
        if (n2 == 0) continue;
        const double kn = sqrt((double)n2);
        const int bin = (int)floor(kn - 0.5);
        if (bin < 0 || bin >= nbins) continue;
        const double w = (iz == 0 || iz == n / 2) ? 1.0 : 2.0;
        const float2 d = c0[m];
        const double p2 = (double)d.x * d.x + (double)d.y * d.y;
        atomicAdd(&sh[3 * bin], w);
        atomicAdd(&sh[3 * bin + 1], w * kn);
        atomicAdd(&sh[3 * bin + 2], w * p2);
    }
    __syncthreads();
    double *dst = acc + (int64_t)b * 3 * nbins;
    for (int q = threadIdx.x; q < 3 * nbins; q += blockDim.x)
        if (sh[q] != 0.0) atomicAdd(dst + q, sh[q]);
}

// ------------------------------------------------------------ white noise --

// Philox4x32-10 (Salmon et al. 2011) with the published multipliers and
// Weyl key increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__global__ void k_noise(const float *noise, uint64_t seed, MeshRef dst, int np) {
    const int b = blockIdx.y;
    const int64_t n3 = (int64_t)np * np * np;
    const uint64_t key = seed + (uint64_t)b;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        float v;
        if (noise) {
            v = noise[(int64_t)b * n3 + i];
        } else {
            const uint4 r = philox4x32_10(make_uint4((unsigned)i, (unsigned)((uint64_t)i >> 32), 0u, 0u),
                                          make_uint2((unsigned)key, (unsigned)(key >> 32)));
            const double u1 = ((double)r.x + 0.5) * 2.3283064365386963e-10;
            const double u2 = ((double)r.y + 0.5) * 2.3283064365386963e-10;
            v = (float)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
        }
        const int64_t row = i / np;
        dst.ptr[(int64_t)b * dst.bstride + row * dst.zs + (i - row * np)] = v;
    }
}

// ------------------------------------------------------------------ 2LPT --

__device__ __forceinline__ double bbks_t(double q) {
    const double x = 2.34 * q;
    const double lead = x > 1e-8 ? log1p(x) / x : 1.0 - 0.5 * x;
    const double a = 16.1 * q, b = 5.46 * q, c = 6.71 * q;
    const double poly = 1.0 + 3.89 * q + a * a + b * b * b + (c * c) * (c * c);
    return lead * rsqrt(sqrt(poly));
}

// d ln T / d ln q of the BBKS form.
__device__ __forceinline__ double bbks_dlnt_dlnq(double q) {
    const double x = 2.34 * q;
    const double dlead = x > 1e-6 ? x / ((1.0 + x) * log1p(x)) - 1.0 : -0.5 * x;
    const double a = 16.1 * q, b = 5.46 * q, c = 6.71 * q;
    const double poly = 1.0 + 3.89 * q + a * a + b * b * b + (c * c) * (c * c);
    const double qdpoly = 3.89 * q + 2.0 * a * a + 3.0 * b * b * b + 4.0 * (c * c) * (c * c);
    return dlead - 0.25 * qdpoly / poly;
}

// sqrt(P(k) / V_c) (m) and its d/dOm (dm) for |k| in h/Mpc.
__device__ __forceinline__ void linear_mult(double k, const LinParams &lp, double &m, double &dm) {
    if (k <= 0.0) {
        m = dm = 0.0;
        return;
    }
    const double q = k / (lp.om * lp.h);
    const double t = bbks_t(q);
    const double pk = lp.amp * pow(k, lp.ns) * t * t;
    m = sqrt(pk * lp.inv_vc);
    const double dlnp = lp.dlnamp - 2.0 * bbks_dlnt_dlnq(q) / lp.om;
    dm = 0.5 * m * dlnp;
}

// omega(k) in field 0 -> s1_j (fields 0..2) and phi_ij (fields 3..8:
// xx, yy, zz, xy, xz, yz), all scaled by 1/n^3 for the inverse transform.
__global__ void __launch_bounds__(kThreads) k_lpt_linear(Spec sp, const LinParams *lps) {
    const int b = blockIdx.y;
    const int n = sp.n;
    const int64_t nmodes = (int64_t)n * n * sp.zc;
    const int64_t m = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (m >= nmodes) return;
    int ix, iy, iz;
    mode_ijk(m, n, sp.zc, sp.blk, ix, iy, iz);
    if (iz > n / 2) return;
    const double kx = sp.kf * (double)signed_index(ix, n), ky = sp.kf * (double)signed_index(iy, n),
                 kz = sp.kf * (double)iz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    double ml, dml;
    linear_mult(sqrt(k2), lps[b], ml, dml);
    float2 *c0 = sp.c + (int64_t)b * sp.bstride + m;
    const int64_t fs = sp.fstride;
    const float2 w = c0[0];
    const double inv = k2 > 0.0 ? ml / (k2 * (double)n * n * n) : 0.0;
    const double dx = w.x * inv, dy = w.y * inv;  // delta_L / (k^2 n^3)
    const int h = n / 2;
    const bool nx = ix == h, ny = iy == h, nz = iz == h;
    const double k[3] = {kx, ky, kz};
    const bool ny3[3] = {nx, ny, nz};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double a = ny3[j] ? 0.0 : k[j];
        c0[j * fs] = make_float2((float)(-a * dy), (float)(a * dx));
    }
    const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const bool zero = (pi[q] != pj[q]) && (ny3[pi[q]] || ny3[pj[q]]);
        const double a = zero ? 0.0 : k[pi[q]] * k[pj[q]];
        c0[(3 + q) * fs] = make_float2((float)(a * dx), (float)(a * dy));
    }
}

// S = phi_xx phi_yy + phi_xx phi_zz + phi_yy phi_zz - phi_xy^2 - phi_xz^2 - phi_yz^2
__global__ void k_lpt_source(MeshRef lat, int np, int f_phi, int f_src) {
    const int b = blockIdx.y;
    const int64_t n3 = (int64_t)np * np * np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / np;
        const int64_t o = (int64_t)b * lat.bstride + row * lat.zs + (i - row * np);
        const float *ph = lat.ptr + f_phi * lat.fstride + o;
        const float xx = ph[0], yy = ph[lat.fstride], zz = ph[2 * lat.fstride];
        const float xy = ph[3 * lat.fstride], xz = ph[4 * lat.fstride], yz = ph[5 * lat.fstride];
        lat.ptr[f_src * lat.fstride + o] = xx * yy + xx * zz + yy * zz - xy * xy - xz * xz - yz * yz;
    }
}

// out_j = sign * i k_j / k^2 * S(k) / n^3 (Nyquist along j zero)
__global__ void __launch_bounds__(kThreads) k_lpt_second(Spec sp, int f_src, int f_out, float sign) {
    const int b = blockIdx.y;
    const int n = sp.n;
    const int64_t nmodes = (int64_t)n * n * sp.zc;
    const int64_t m = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (m >= nmodes) return;
    int ix, iy, iz;
    mode_ijk(m, n, sp.zc, sp.blk, ix, iy, iz);
    if (iz > n / 2) return;
    const float kx = sp.kf * signed_index(ix, n), ky = sp.kf * signed_index(iy, n), kz = sp.kf * iz;
    const float k2 = kx * kx + ky * ky + kz * kz;
    const float g = k2 > 0.f ? sign / (k2 * (float)n * n * n) : 0.f;
    float2 *c0 = sp.c + (int64_t)b * sp.bstride + m;
    const float2 s = c0[f_src * sp.fstride];
    const int h = n / 2;
    c0[f_out * sp.fstride] = times_i(s, ix == h ? 0.f : kx * g);
    c0[(f_out + 1) * sp.fstride] = times_i(s, iy == h ? 0.f : ky * g);
    c0[(f_out + 2) * sp.fstride] = times_i(s, iz == h ? 0.f : kz * g);
}

// Adjoint of k_lpt_second with sign -1: S_bar(k) = sum_j (+i k_j / k^2) G_j(k) / n^3.
__global__ void __launch_bounds__(kThreads) k_lpt_adj_second(Spec sp, int f_in, int f_out) {
    const int b = blockIdx.y;
    const int n = sp.n;
    const int64_t nmodes = (int64_t)n * n * sp.zc;
    const int64_t m = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (m >= nmodes) return;
    int ix, iy, iz;
    mode_ijk(m, n, sp.zc, sp.blk, ix, iy, iz);
    if (iz > n / 2) return;
    const float kx = sp.kf * signed_index(ix, n), ky = sp.kf * signed_index(iy, n), kz = sp.kf * iz;
    const float k2 = kx * kx + ky * ky + kz * kz;
    const float g = k2 > 0.f ? 1.f / (k2 * (float)n * n * n) : 0.f;
    float2 *c0 = sp.c + (int64_t)b * sp.bstride + m;
    const int h = n / 2;
    const float2 a = times_i(c0[f_in * sp.fstride], ix == h ? 0.f : kx * g);
    const float2 bb = times_i(c0[(f_in + 1) * sp.fstride], iy == h ? 0.f : ky * g);
    const float2 c = times_i(c0[(f_in + 2) * sp.fstride], iz == h ? 0.f : kz * g);
    c0[f_out * sp.fstride] = make_float2(a.x + bb.x + c.x, a.y + bb.y + c.y);
}

__device__ __forceinline__ int64_t lat_off(const MeshRef &lat, int b, int64_t i, int np) {
    const int64_t row = i / np;
    return (int64_t)b * lat.bstride + row * lat.zs + (i - row * np);
}

// s = D1 s1 + D2 s2, p = g1 s1 + g2 s2 (s1 in fields 0..2, s2 in 10..12).
__global__ void k_lpt_combine(MeshRef lat, int np, const float4 *fac, float *s, float *p) {
    const int b = blockIdx.y;
    const int64_t n3 = (int64_t)np * np * np;
    const float4 c = fac[b];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = lat_off(lat, b, i, np);
        const int64_t gi = ((int64_t)b * n3 + i) * 3;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float a1 = lat.ptr[j * lat.fstride + o];
            const float a2 = lat.ptr[(10 + j) * lat.fstride + o];
            s[gi + j] = c.x * a1 + c.y * a2;
            p[gi + j] = c.z * a1 + c.w * a2;
        }
    }
}

// Reductions (lam.s1, lam.s2, mu.s1, mu.s2) per batch and cotangents
// gs1 = D1 lam + g1 mu -> fields 0..2, gs2 = D2 lam + g2 mu -> fields 10..12.
__global__ void __launch_bounds__(kThreads) k_lpt_adj_seed(MeshRef lat, int np, const float4 *fac, const float *lam,
                                                           const float *mu, double *red) {
    const int b = blockIdx.y;
    const int64_t n3 = (int64_t)np * np * np;
    const float4 c = fac[b];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = lat_off(lat, b, i, np);
        const int64_t gi = ((int64_t)b * n3 + i) * 3;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float l = lam[gi + j], u = mu[gi + j];
            float *f1 = lat.ptr + j * lat.fstride + o;
            float *f2 = lat.ptr + (10 + j) * lat.fstride + o;
            const float a1 = *f1, a2 = *f2;
            acc[0] += (double)(l * a1);
            acc[1] += (double)(l * a2);
            acc[2] += (double)(u * a1);
            acc[3] += (double)(u * a2);
            *f1 = c.x * l + c.z * u;
            *f2 = c.y * l + c.w * u;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double v = acc[q];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(red + 4 * b + q, v);
    }
}

// phi_bar from S_bar (field 9) and phi (fields 3..8), in place over phi.
__global__ void k_lpt_adj_phi(MeshRef lat, int np) {
    const int b = blockIdx.y;
    const int64_t n3 = (int64_t)np * np * np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = lat_off(lat, b, i, np);
        const int64_t fs = lat.fstride;
        float *ph = lat.ptr + 3 * fs + o;
        const float sb = lat.ptr[9 * fs + o];
        const float xx = ph[0], yy = ph[fs], zz = ph[2 * fs], xy = ph[3 * fs], xz = ph[4 * fs], yz = ph[5 * fs];
        ph[0] = sb * (yy + zz);
        ph[fs] = sb * (xx + zz);
        ph[2 * fs] = sb * (xx + yy);
        ph[3 * fs] = -2.f * sb * xy;
        ph[4 * fs] = -2.f * sb * xz;
        ph[5 * fs] = -2.f * sb * yz;
    }
}

// delta_bar(k) = sum_j conj(i k_j / k^2) G1_j + sum_q m_q Phi_bar_q from
// fields 0..8; omega_bar(k) = m_lin delta_bar / n^3 -> field 0; reductions
// red[b][0] += w Re(conj(delta_bar) m_lin omega), red[b][1] the same with
// d m_lin / dOm (Parseval; scaled by 1/n^3 on the host).
__global__ void __launch_bounds__(kThreads) k_lpt_adj_final(Spec sp, const LinParams *lps, int f_noise, double *red) {
    const int b = blockIdx.y;
    const int n = sp.n;
    const int64_t nmodes = (int64_t)n * n * sp.zc;
    const int64_t m = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    double r0 = 0.0, r1 = 0.0;
    int ix = 0, iy = 0, iz = 0;
    if (m < nmodes) mode_ijk(m, n, sp.zc, sp.blk, ix, iy, iz);
    if (m < nmodes && iz <= n / 2) {
        const double kx = sp.kf * (double)signed_index(ix, n), ky = sp.kf * (double)signed_index(iy, n),
                     kz = sp.kf * (double)iz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        double ml, dml;
        linear_mult(sqrt(k2), lps[b], ml, dml);
        float2 *c0 = sp.c + (int64_t)b * sp.bstride + m;
        const int64_t fs = sp.fstride;
        const int h = n / 2;
        const bool nyq[3] = {ix == h, iy == h, iz == h};
        const double k[3] = {kx, ky, kz};
        const double inv = k2 > 0.0 ? 1.0 / k2 : 0.0;
        double ax = 0.0, ay = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double a = nyq[j] ? 0.0 : -k[j] * inv;  // conj(i k_j / k^2) = -i k_j / k^2
            const float2 g = c0[j * fs];
            ax += -a * g.y;
            ay += a * g.x;
        }
        const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const bool zero = (pi[q] != pj[q]) && (nyq[pi[q]] || nyq[pj[q]]);
            const double a = zero ? 0.0 : k[pi[q]] * k[pj[q]] * inv;
            const float2 g = c0[(3 + q) * fs];
            ax += a * g.x;
            ay += a * g.y;
        }
        const float2 w = c0[f_noise * fs];
        const double wt = (iz == 0 || iz == h) ? 1.0 : 2.0;
        r0 = wt * ml * (ax * w.x + ay * w.y);
        r1 = wt * dml * (ax * w.x + ay * w.y);
        const double sc = ml / ((double)n * n * n);
        c0[0] = make_float2((float)(sc * ax), (float)(sc * ay));
    }
    for (int o = 16; o; o >>= 1) {
        r0 += __shfl_xor_sync(0xffffffffu, r0, o);
        r1 += __shfl_xor_sync(0xffffffffu, r1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red + 2 * b, r0);
        atomicAdd(red + 2 * b + 1, r1);
    }
}

template <int T>
void spectral_t(int mode, const Spec &sp, const float *pref, cudaStream_t st) {
    const int64_t nmodes = (int64_t)sp.n * sp.n * sp.zc;
    const dim3 grid((unsigned)((nmodes + T - 1) / T), sp.nb);
    if (mode == SPEC_FORCE)
        k_spec_force<T><<<grid, T, 0, st>>>(sp, pref);
    else
        k_spec_adj<T><<<grid, T, 0, st>>>(sp, pref);
}

dim3 mode_grid(const Spec &sp) {
    const int64_t nmodes = (int64_t)sp.n * sp.n * sp.zc;
    return dim3((unsigned)((nmodes + kThreads - 1) / kThreads), sp.nb);
}

dim3 site_grid(int np, int nb) {
    const int64_t n3 = (int64_t)np * np * np;
    const int64_t blocks = (n3 + kThreads - 1) / kThreads;
    return dim3((unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), nb);
}

// The force from the potential mesh: F_j(c) = S_j phi(c), S_j the periodic
// 4-point central difference along axis j,
//   S f(c) = [8 (f(c + e_j) - f(c - e_j)) - (f(c + 2 e_j) - f(c - 2 e_j))] / (12 h),
// whose Fourier symbol is i D_j (zero at the Nyquist index exactly: the two
// differences of an alternating line vanish).  in: planar [gi][run][n^3],
// phi (and psi when GI = 2); out: [run][n^3] float4 (F_x, F_y, F_z, psi or
// 0), the layout the read kernels take.  n is a power of two (own-FFT
// meshes).  A block takes a TX x TY x TZ tile: the tile and a 2-node
// periodic halo of phi go to shared memory in coalesced rows along z, every
// thread then forms its nodes' three differences from shared memory.  Tiles
// run z fastest, then y, then x, so neighbouring blocks share halo lines in L2.
template <int GI, int TZ>
__global__ void __launch_bounds__(kThreads) k_grad_stencil(const float *__restrict__ in, float4 *__restrict__ out,
                                                           int lgn, float inv12h) {
    constexpr int TX = 4, TY = 4, HX = TX + 4, HY = TY + 4, HZ = TZ + 4;
    constexpr int PER = TX * TY * TZ / kThreads;
    __shared__ float tile[HX][HY][HZ];
    const int n = 1 << lgn, m = n - 1;
    const int64_t n3 = (int64_t)1 << (3 * lgn);
    const int b = blockIdx.y;
    const float *phi = in + (int64_t)b * n3;
    const int ntz = n / TZ, nty = n / TY;
    const int t = blockIdx.x;
    const int z0 = (t % ntz) * TZ, y0 = ((t / ntz) % nty) * TY, x0 = (t / ntz / nty) * TX;
    for (int e = threadIdx.x; e < HX * HY * HZ; e += kThreads) {
        const int iz = e % HZ, iy = (e / HZ) % HY, ix = e / (HZ * HY);
        const int64_t g = (((int64_t)((x0 + ix - 2) & m) << lgn | ((y0 + iy - 2) & m)) << lgn) | ((z0 + iz - 2) & m);
        tile[ix][iy][iz] = __ldg(phi + g);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int c = threadIdx.x + q * kThreads;
        const int lz = c % TZ, ly = (c / TZ) % TY, lx = c / (TZ * TY);
        const int X = lx + 2, Yy = ly + 2, Z = lz + 2;
        const float fx = inv12h * (8.f * (tile[X + 1][Yy][Z] - tile[X - 1][Yy][Z]) - (tile[X + 2][Yy][Z] - tile[X - 2][Yy][Z]));
        const float fy = inv12h * (8.f * (tile[X][Yy + 1][Z] - tile[X][Yy - 1][Z]) - (tile[X][Yy + 2][Z] - tile[X][Yy - 2][Z]));
        const float fz = inv12h * (8.f * (tile[X][Yy][Z + 1] - tile[X][Yy][Z - 1]) - (tile[X][Yy][Z + 2] - tile[X][Yy][Z - 2]));
        const int64_t g = (((int64_t)(x0 + lx) << lgn | (y0 + ly)) << lgn) | (z0 + lz);
        out[(int64_t)b * n3 + g] = make_float4(fx, fy, fz, GI == 2 ? __ldg(in + (int64_t)gridDim.y * n3 + (int64_t)b * n3 + g) : 0.f);
    }
}

// The adjoint's source on the real mesh: from the 4-field paint (alpha sum W,
// sum mu_x W, sum mu_y W, sum mu_z W) per cell, v = sum_j S_j u_j, S_j the
// periodic 4-point difference along axis j.  Its transform is
// sum_j i D_j u_j(k), so psi(k) = -g v(k) needs one forward transform
// instead of three.  out: [run][n^3] float2 (rho, v).  A block takes a
// 4 x 8 x TZ tile; each component is staged in shared memory with the halo
// of its own axis only (u_x two planes each side in x, u_y two rows in y,
// u_z two nodes in z).
template <int TZ>
__global__ void __launch_bounds__(kThreads) k_vjp_source(const float4 *__restrict__ in, float2 *__restrict__ out,
                                                         int lgn, float inv12h) {
    constexpr int TX = 4, TY = 8, PER = TX * TY * TZ / kThreads;
    __shared__ float ux[TX + 4][TY][TZ], uy[TX][TY + 4][TZ], uz[TX][TY][TZ + 4], rho[TX][TY][TZ];
    const int n = 1 << lgn, m = n - 1;
    const int64_t n3 = (int64_t)1 << (3 * lgn);
    const int b = blockIdx.y;
    const float4 *src = in + (int64_t)b * n3;
    const float *srcf = reinterpret_cast<const float *>(src);
    const int ntz = n / TZ, nty = n / TY;
    const int t = blockIdx.x;
    const int z0 = (t % ntz) * TZ, y0 = ((t / ntz) % nty) * TY, x0 = (t / ntz / nty) * TX;
    auto cell = [&](int x, int y, int z) -> int64_t {
        return (((int64_t)(x & m) << lgn) | (y & m)) << lgn | (z & m);
    };
    // the x-extended block: whole cells inside, u_x alone in the x halo
    for (int e = threadIdx.x; e < (TX + 4) * TY * TZ; e += kThreads) {
        const int iz = e % TZ, iy = (e / TZ) % TY, ix = e / (TZ * TY) - 2;
        if (ix >= 0 && ix < TX) {
            const float4 c = __ldg(src + cell(x0 + ix, y0 + iy, z0 + iz));
            rho[ix][iy][iz] = c.x;
            ux[ix + 2][iy][iz] = c.y;
            uy[ix][iy + 2][iz] = c.z;
            uz[ix][iy][iz + 2] = c.w;
        } else {
            ux[ix + 2][iy][iz] = __ldg(srcf + 4 * cell(x0 + ix, y0 + iy, z0 + iz) + 1);
        }
    }
    for (int e = threadIdx.x; e < TX * 4 * TZ; e += kThreads) {  // y halo: u_y
        const int iz = e % TZ, q = (e / TZ) % 4, ix = e / (TZ * 4);
        const int iy = q < 2 ? q - 2 : TY + q - 2;
        uy[ix][iy + 2][iz] = __ldg(srcf + 4 * cell(x0 + ix, y0 + iy, z0 + iz) + 2);
    }
    for (int e = threadIdx.x; e < TX * TY * 4; e += kThreads) {  // z halo: u_z
        const int q = e % 4, iy = (e / 4) % TY, ix = e / (4 * TY);
        const int iz = q < 2 ? q - 2 : TZ + q - 2;
        uz[ix][iy][iz + 2] = __ldg(srcf + 4 * cell(x0 + ix, y0 + iy, z0 + iz) + 3);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int c = threadIdx.x + q * kThreads;
        const int lz = c % TZ, ly = (c / TZ) % TY, lx = c / (TZ * TY);
        const float sx = 8.f * (ux[lx + 3][ly][lz] - ux[lx + 1][ly][lz]) - (ux[lx + 4][ly][lz] - ux[lx][ly][lz]);
        const float sy = 8.f * (uy[lx][ly + 3][lz] - uy[lx][ly + 1][lz]) - (uy[lx][ly + 4][lz] - uy[lx][ly][lz]);
        const float sz = 8.f * (uz[lx][ly][lz + 3] - uz[lx][ly][lz + 1]) - (uz[lx][ly][lz + 4] - uz[lx][ly][lz]);
        const int64_t g = (((int64_t)(x0 + lx) << lgn | (y0 + ly)) << lgn) | (z0 + lz);
        out[(int64_t)b * n3 + g] = make_float2(rho[lx][ly][lz], inv12h * (sx + sy + sz));
    }
}

// The same source for meshes of 64 and more per side, marching along x: a
// block owns an 8 (y) x 32 (z) patch of cells, one thread a (y, z) column
// (warp = y row, lane = z), and walks XC planes x0 .. x0 + XC - 1 with two
// planes of halo on either side, so u_x of a cell is loaded once per block
// instead of once per tile and its four x neighbours flow through a
// five-register window.  Per plane: the cell's float4 (next plane's loads
// issued while this one is processed), u_y of the 8 rows plus the two halo
// rows each side through a double-buffered shared-memory plane (one barrier
// per plane), u_z of the z neighbours by warp shuffles (lanes 0..3 fetch the
// four halo nodes).  S_y u_y + S_z u_z of plane x waits two planes, until
// u_x of plane x + 2 has arrived.
template <int XC>
__global__ void __launch_bounds__(kThreads) k_vjp_source_x(const float4 *__restrict__ in, float2 *__restrict__ out,
                                                           int lgn, float inv12h) {
    constexpr int TY = kThreads / 32;
    __shared__ float uys[2][TY + 4][32];
    const int n = 1 << lgn, m = n - 1;
    const int64_t n3 = (int64_t)1 << (3 * lgn);
    const int b = blockIdx.y;
    const float4 *src = in + (int64_t)b * n3;
    const float *srcf = reinterpret_cast<const float *>(src);
    float2 *dst = out + (int64_t)b * n3;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nz = n / 32, ny = n / TY;
    const int t = blockIdx.x;
    const int z0 = (t % nz) * 32, y0 = ((t / nz) % ny) * TY, x0 = (t / nz / ny) * XC;
    const int y = y0 + w, z = z0 + lane;
    auto cell = [&](int xx, int yy, int zz) -> int64_t {
        return (((int64_t)(xx & m) << lgn) | (yy & m)) << lgn | (zz & m);
    };
    // halo fetches of plane xx: warps 0..3 the u_y rows y0 - 2, y0 - 1, y0 + TY, y0 + TY + 1;
    // lanes 0..3 the u_z nodes z0 - 2, z0 - 1, z0 + 32, z0 + 33 of their row
    const int hy = w < 2 ? y0 - 2 + w : y0 + TY + w - 2;
    const int hz = lane < 2 ? z0 - 2 + lane : z0 + 30 + lane;
    float ux[5] = {0.f, 0.f, 0.f, 0.f, 0.f};                  // u_x at planes p - 4 .. p of this column
    float vq[3] = {0.f, 0.f, 0.f}, rq[3] = {0.f, 0.f, 0.f};  // S_y u_y + S_z u_z and rho of planes p - 2 .. p
    float4 cur = make_float4(0.f, 0.f, 0.f, 0.f);
    float cur_hy = 0.f, cur_hz = 0.f;
    auto fetch = [&](int p, float4 &c, float &fy, float &fz) {
        const bool inner = p >= x0 && p < x0 + XC;
        if (inner) {
            c = __ldg(src + cell(p, y, z));
            if (w < 4) fy = __ldg(srcf + 4 * cell(p, hy, z) + 2);
            if (lane < 4) fz = __ldg(srcf + 4 * cell(p, y, hz) + 3);
        } else {
            c.y = __ldg(srcf + 4 * cell(p, y, z) + 1);  // u_x alone in the x halo
        }
    };
    fetch(x0 - 2, cur, cur_hy, cur_hz);
    for (int p = x0 - 2; p < x0 + XC + 2; ++p) {
        float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
        float nxt_hy = 0.f, nxt_hz = 0.f;
        if (p + 1 < x0 + XC + 2) fetch(p + 1, nxt, nxt_hy, nxt_hz);
#pragma unroll
        for (int k = 0; k < 4; ++k) ux[k] = ux[k + 1];
        ux[4] = cur.y;
        vq[0] = vq[1];
        vq[1] = vq[2];
        rq[0] = rq[1];
        rq[1] = rq[2];
        if (p >= x0 && p < x0 + XC) {  // uniform across the block
            float(*plane)[32] = uys[p & 1];
            plane[w + 2][lane] = cur.z;
            if (w < 4) plane[w < 2 ? w : TY + w][lane] = cur_hy;
            __syncthreads();
            const float sy = 8.f * (plane[w + 3][lane] - plane[w + 1][lane]) - (plane[w + 4][lane] - plane[w][lane]);
            const float hm2 = __shfl_sync(0xffffffffu, cur_hz, 0), hm1 = __shfl_sync(0xffffffffu, cur_hz, 1);
            const float hp1 = __shfl_sync(0xffffffffu, cur_hz, 2), hp2 = __shfl_sync(0xffffffffu, cur_hz, 3);
            float zm1 = __shfl_up_sync(0xffffffffu, cur.w, 1), zm2 = __shfl_up_sync(0xffffffffu, cur.w, 2);
            float zp1 = __shfl_down_sync(0xffffffffu, cur.w, 1), zp2 = __shfl_down_sync(0xffffffffu, cur.w, 2);
            if (lane == 0) zm1 = hm1;
            if (lane < 2) zm2 = lane == 0 ? hm2 : hm1;
            if (lane == 31) zp1 = hp1;
            if (lane > 29) zp2 = lane == 31 ? hp2 : hp1;
            vq[2] = sy + (8.f * (zp1 - zm1) - (zp2 - zm2));
            rq[2] = cur.x;
        }
        const int q = p - 2;  // ux[0 .. 4] = u_x at q - 2 .. q + 2
        if (q >= x0 && q < x0 + XC) {
            const float sx = 8.f * (ux[3] - ux[1]) - (ux[4] - ux[0]);
            dst[cell(q, y, z)] = make_float2(rq[0], inv12h * (sx + vq[0]));
        }
        cur = nxt;
        cur_hy = nxt_hy;
        cur_hz = nxt_hz;
    }
}

}  // namespace

cudaError_t launch_vjp_source(const float4 *in, float2 *out, int n, int nb, float inv12h, cudaStream_t st) {
    int lgn = 0;
    while ((1 << lgn) < n) ++lgn;
    if ((1 << lgn) != n || n < 16) return cudaErrorInvalidValue;
    if (n >= 64) {  // x-marching blocks of 8 x 32 columns over 64 planes
        constexpr int XC = 64, TY = kThreads / 32;
        k_vjp_source_x<XC><<<dim3((unsigned)((n / 32) * (n / TY) * (n / XC)), nb), kThreads, 0, st>>>(in, out, lgn,
                                                                                                    inv12h);
        return cudaGetLastError();
    }
    const int tz = n < 32 ? n : 32;
    const dim3 grid((unsigned)((n / 4) * (n / 8) * (n / tz)), nb);
    if (tz == 16)
        k_vjp_source<16><<<grid, kThreads, 0, st>>>(in, out, lgn, inv12h);
    else
        k_vjp_source<32><<<grid, kThreads, 0, st>>>(in, out, lgn, inv12h);
    return cudaGetLastError();
}

cudaError_t launch_grad_stencil(const float *in, int gi, float4 *out, int n, int nb, float inv12h, cudaStream_t st) {
    int lgn = 0;
    while ((1 << lgn) < n) ++lgn;
    if ((1 << lgn) != n || n < 16 || (gi != 1 && gi != 2)) return cudaErrorInvalidValue;
    const int tz = n < 128 ? n : 128;
    const dim3 grid((unsigned)((n / 4) * (n / 4) * (n / tz)), nb);
    auto go = [&](auto kernel) { kernel<<<grid, kThreads, 0, st>>>(in, out, lgn, inv12h); };
    switch (tz * 4 + gi) {
        case 16 * 4 + 1: go(k_grad_stencil<1, 16>); break;
        case 16 * 4 + 2: go(k_grad_stencil<2, 16>); break;
        case 32 * 4 + 1: go(k_grad_stencil<1, 32>); break;
        case 32 * 4 + 2: go(k_grad_stencil<2, 32>); break;
        case 64 * 4 + 1: go(k_grad_stencil<1, 64>); break;
        case 64 * 4 + 2: go(k_grad_stencil<2, 64>); break;
        case 128 * 4 + 1: go(k_grad_stencil<1, 128>); break;
        default: go(k_grad_stencil<2, 128>); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_spectral(int mode, const Spec &sp, const float *pref, cudaStream_t st) {
    switch (sp.threads) {
        case 128: spectral_t<128>(mode, sp, pref, st); break;
        case 512: spectral_t<512>(mode, sp, pref, st); break;
        default: spectral_t<256>(mode, sp, pref, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_power_bins(const Spec &sp, double *acc, int nbins, cudaStream_t st) {
    const size_t smem = sizeof(double) * 3 * nbins;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_power_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t nmodes = (int64_t)sp.n * sp.n * sp.zc;
    const int64_t blocks = (nmodes + kThreads - 1) / kThreads;
    k_power_bins<<<dim3((unsigned)(blocks < 152 * 4 ? blocks : 152 * 4), sp.nb), kThreads, smem, st>>>(sp, acc, nbins);
    return cudaGetLastError();
}

cudaError_t launch_noise(const float *noise, uint64_t seed, MeshRef dst, int np, int nb, cudaStream_t st) {
    k_noise<<<site_grid(np, nb), kThreads, 0, st>>>(noise, seed, dst, np);
    return cudaGetLastError();
}

cudaError_t launch_lpt_linear(const Spec &sp, const LinParams *lp, cudaStream_t st) {
    k_lpt_linear<<<mode_grid(sp), kThreads, 0, st>>>(sp, lp);
    return cudaGetLastError();
}

cudaError_t launch_lpt_source(MeshRef lat, int np, int nb, int f_phi, int f_src, cudaStream_t st) {
    k_lpt_source<<<site_grid(np, nb), kThreads, 0, st>>>(lat, np, f_phi, f_src);
    return cudaGetLastError();
}

cudaError_t launch_lpt_second(const Spec &sp, int f_src, int f_out, float sign, cudaStream_t st) {
    k_lpt_second<<<mode_grid(sp), kThreads, 0, st>>>(sp, f_src, f_out, sign);
    return cudaGetLastError();
}

cudaError_t launch_lpt_adj_second(const Spec &sp, int f_in, int f_out, cudaStream_t st) {
    k_lpt_adj_second<<<mode_grid(sp), kThreads, 0, st>>>(sp, f_in, f_out);
    return cudaGetLastError();
}

cudaError_t launch_lpt_combine(MeshRef lat, int np, int nb, const float4 *fac, float *s, float *p, cudaStream_t st) {
    k_lpt_combine<<<site_grid(np, nb), kThreads, 0, st>>>(lat, np, fac, s, p);
    return cudaGetLastError();
}

cudaError_t launch_lpt_adj_seed(MeshRef lat, int np, int nb, const float4 *fac, const float *lam, const float *mu,
                                double *red, cudaStream_t st) {
    k_lpt_adj_seed<<<site_grid(np, nb), kThreads, 0, st>>>(lat, np, fac, lam, mu, red);
    return cudaGetLastError();
}

cudaError_t launch_lpt_adj_phi(MeshRef lat, int np, int nb, cudaStream_t st) {
    k_lpt_adj_phi<<<site_grid(np, nb), kThreads, 0, st>>>(lat, np);
    return cudaGetLastError();
}

cudaError_t launch_lpt_adj_final(const Spec &sp, const LinParams *lp, int f_noise, double *red, cudaStream_t st) {
    k_lpt_adj_final<<<mode_grid(sp), kThreads, 0, st>>>(sp, lp, f_noise, red);
    return cudaGetLastError();
}

}  // namespace pmgb
