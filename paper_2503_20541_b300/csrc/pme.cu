// pme.cu -- smooth particle-mesh Ewald, order 4 (Sec. 2.1.2; Essmann et al. 1995).
//
//   spread   : Q(k) = sum_i q_i M4(u_i0 - k0) M4(u_i1 - k1) M4(u_i2 - k2), u_d = K_d x_d / L_d,
//              accumulated with int64 fixed-point atomics (order-independent, so the
//              mesh is bitwise reproducible), then converted to FP32 for cuFFT.
//   convolve : Q^(m) *= G(m), G = ke/(pi V) exp(-pi^2 |m|^2 / alpha^2) / |m|^2 B(m),
//              E_rec = 1/2 sum_m G |Q^(m)|^2 over the full spectrum (half spectrum
//              weighted 2 for the interior k2 columns), summed in FP64 per block.
//   gather   : F_i = -q_i sum_k grad_i[M4 M4 M4](k) phi(k), phi = c2r(G Q^) (unnormalised).
// The order-4 weights use the closed-form cubic pieces of M4 on [0,1], [1,2], [2,3], [3,4].
// cuFFT performs the 3-D transforms (one batched plan per distinct mesh shape).
#include <climits>
#include <math.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace nb {

// Order-4 B-spline weights w[j] = M4(t + j) for grid point floor(u) - j, and dw[j] = dM4/du.
__device__ __forceinline__ void bspline4(float t, float w[4], float dw[4]) {
    float t2 = t * t, t3 = t2 * t;
    float s = 1.f - t;
    const float c6 = 1.f / 6.f;
    w[0] = t3 * c6;
    w[1] = (-3.f * t3 + 3.f * t2 + 3.f * t + 1.f) * c6;
    w[2] = (3.f * t3 - 6.f * t2 + 4.f) * c6;
    w[3] = s * s * s * c6;
    dw[0] = 0.5f * t2;
    dw[1] = 0.5f * (-3.f * t2 + 2.f * t + 1.f);
    dw[2] = 0.5f * (3.f * t2 - 4.f * t);
    dw[3] = -0.5f * s * s;
}

// Fractional mesh coordinate u = x K/L split into floor and fraction.  K/L is held as
// hi + lo and the product's rounding error is recovered with an FMA, so t keeps full
// FP32 accuracy even where u ~ K (a plain FP32 product loses ~log2(K) bits of t).
__device__ __forceinline__ void frac_coord(float x, int K, float kh, float kl, int& fl, float& t) {
    float u = x * kh;
    float err = fmaf(x, kh, -u) + x * kl;
    float f = floorf(u);
    t = (u - f) + err;
    if (t >= 1.f) {
        t -= 1.f;
        f += 1.f;
    }
    if (t < 0.f) {
        t += 1.f;
        f -= 1.f;
    }
    fl = (int)f;
    if ((unsigned)fl >= (unsigned)K) {  // caller coordinates may lie several boxes away
        fl %= K;
        if (fl < 0) fl += K;
    }
}

__device__ __forceinline__ int wrapk(int k, int K) { return k < 0 ? k + K : k; }

// v[j] for a run-time j in 0..3 by selects, so that v stays in registers (an indexed
// array would be placed in local memory).
__device__ __forceinline__ float pick4(const float v[4], int j) {
    float r = v[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) r = j == k ? v[k] : r;
    return r;
}

// 16 threads per atom: thread (b, c) owns y offset b and z offset c and visits the 4 x
// offsets, so that each warp-wide atomic covers 8 runs of 4 consecutive mesh points (z is
// the contiguous axis).  The positions may be in either order (caller or slot): the mesh
// sums are order-free.
__global__ void k_spread(int N, const float4* __restrict__ xs, const int* __restrict__ sid,
                         const SysDev* __restrict__ sys, long long* __restrict__ gfix, float gscale) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt >> 4, sub = gt & 15;
    if (i >= N) return;
    const SysDev& S = sys[sid[i]];
    if (!S.pme) return;
    float4 p = xs[i];
    int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
    int f0, f1, f2;
    float t0, t1, t2;
    frac_coord(p.x, K0, S.kl_hi[0], S.kl_lo[0], f0, t0);
    frac_coord(p.y, K1, S.kl_hi[1], S.kl_lo[1], f1, t1);
    frac_coord(p.z, K2, S.kl_hi[2], S.kl_lo[2], f2, t2);
    float w0[4], w1[4], w2[4], d[4];
    bspline4(t0, w0, d);
    bspline4(t1, w1, d);
    bspline4(t2, w2, d);
    const int b = sub >> 2, c = sub & 3;
    const int iy = wrapk(f1 - b, K1), iz = wrapk(f2 - c, K2);
    const float wyz = p.w * pick4(w1, b) * pick4(w2, c);
    long long* g = gfix + S.grid_off + (long long)iy * K2 + iz;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int ix = wrapk(f0 - a, K0);
        red_add(g + (long long)ix * K1 * K2, __float2ll_rn(w0[a] * wyz * gscale));
    }
}

__global__ void k_grid_convert(long long n, long long* __restrict__ gfix, float* __restrict__ grid, double ginv) {
    pdl_wait();
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    grid[k] = (float)((double)gfix[k] * ginv);
    gfix[k] = 0;
}

// Influence function (FP64, once at set-up).
__global__ void k_green(int K0, int K1, int K2, double L0, double L1, double L2, double alpha, double ke,
                        float* __restrict__ green) {
    int K2h = K2 / 2 + 1;
    long long n = (long long)K0 * K1 * K2h;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int k2 = (int)(c % K2h);
    int k1 = (int)((c / K2h) % K1);
    int k0 = (int)(c / ((long long)K2h * K1));
    if (k0 == 0 && k1 == 0 && k2 == 0) {
        green[c] = 0.f;
        return;
    }
    const double pi = 3.14159265358979323846;
    double m0 = (k0 <= K0 / 2 ? k0 : k0 - K0) / L0;
    double m1 = (k1 <= K1 / 2 ? k1 : k1 - K1) / L1;
    double m2 = k2 / L2;
    double m2s = m0 * m0 + m1 * m1 + m2 * m2;
    // |b(k)|^2 = 1 / |sum_{j=0}^{2} M4(j+1) exp(2 pi i k j / K)|^2 with M4(1..3) = 1/6, 2/3, 1/6
    auto bmod = [&](int k, int K) {
        double th = 2.0 * pi * k / K;
        double re = 1.0 / 6.0 + 2.0 / 3.0 * cos(th) + 1.0 / 6.0 * cos(2.0 * th);
        double im = 2.0 / 3.0 * sin(th) + 1.0 / 6.0 * sin(2.0 * th);
        return 1.0 / (re * re + im * im);
    };
    double V = L0 * L1 * L2;
    double G = ke / (pi * V) * exp(-pi * pi * m2s / (alpha * alpha)) / m2s * bmod(k0, K0) * bmod(k1, K1) *
               bmod(k2, K2);
    green[c] = (float)G;
}

constexpr int kConvThreads = 256;
constexpr int kConvItems = 2;
constexpr int kConvTile = kConvThreads * kConvItems;

__global__ void __launch_bounds__(kConvThreads) k_convolve(const int* __restrict__ blk_sys,
                                                           const int* __restrict__ blk_off,
                                                           const SysDev* __restrict__ sys,
                                                           float2* __restrict__ cgrid,
                                                           const float* __restrict__ green,
                                                           double* __restrict__ e_blk) {
    pdl_wait();
    int b = blockIdx.x;
    int s = blk_sys[b];
    const SysDev& S = sys[s];
    int K2h = S.K[2] / 2 + 1;
    long long n = (long long)S.K[0] * S.K[1] * K2h;
    long long base = (long long)(b - blk_off[s]) * kConvTile;
    float acc = 0.f;
#pragma unroll
    for (int it = 0; it < kConvItems; ++it) {
        long long c = base + it * kConvThreads + threadIdx.x;
        if (c < n) {
            // 32-bit remainder when the mesh allows it (a 64-bit one is a long software sequence)
            int k2 = n <= INT_MAX ? (int)c % K2h : (int)(c % K2h);
            float g = green[S.cgrid_off + c];
            float2 q = cgrid[S.cgrid_off + c];
            float mult = (k2 == 0 || (2 * k2 == S.K[2])) ? 1.f : 2.f;
            acc = fmaf(0.5f * mult * g, q.x * q.x + q.y * q.y, acc);
            cgrid[S.cgrid_off + c] = make_float2(q.x * g, q.y * g);
        }
    }
    if (!e_blk) return;  // convolution only (the VJP's second mesh)
    double v = (double)acc;
    __shared__ double red[kConvThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kConvThreads / 32; ++w) t += red[w];
        e_blk[b] = t;
    }
}

// 16 lanes per atom; mode 0 adds -q grad into ffix (slot order, atomically; atom i of xs
// goes to slot slot_of[i], or to slot i when slot_of is null), mode 1 writes f_out (caller
// order; xs in slot order).
__global__ void k_gather(int N, const float4* __restrict__ xs, const int* __restrict__ sid,
                         const SysDev* __restrict__ sys, const float* __restrict__ phi,
                         long long* __restrict__ ffix, float* __restrict__ f_out, const int* __restrict__ perm,
                         const int* __restrict__ slot_of, float scale, int mode, unsigned* flags) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt >> 4, sub = gt & 15;
    bool valid = i < N;
    int ii = valid ? i : N - 1;
    const SysDev& S = sys[sid[ii]];
    bool pme = valid && S.pme;
    float gxs = 0.f, gys = 0.f, gzs = 0.f;
    float q = 0.f;
    float k0l = 0.f, k1l = 0.f, k2l = 0.f;
    if (pme) {
        float4 p = xs[ii];
        q = p.w;
        int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
        k0l = S.kl_hi[0];
        k1l = S.kl_hi[1];
        k2l = S.kl_hi[2];
        int f0, f1, f2;
        float t0, t1, t2;
        frac_coord(p.x, K0, S.kl_hi[0], S.kl_lo[0], f0, t0);
        frac_coord(p.y, K1, S.kl_hi[1], S.kl_lo[1], f1, t1);
        frac_coord(p.z, K2, S.kl_hi[2], S.kl_lo[2], f2, t2);
        float w0[4], w1[4], w2[4], d0[4], d1[4], d2[4];
        bspline4(t0, w0, d0);
        bspline4(t1, w1, d1);
        bspline4(t2, w2, d2);
        // lane (b, c) of the atom's 16: y offset b, z offset c, the 4 x offsets in turn (each
        // warp-wide load covers 8 runs of 4 consecutive mesh points)
        const int b = sub >> 2, c = sub & 3;
        const int iy = wrapk(f1 - b, K1), iz = wrapk(f2 - c, K2);
        const float* g = phi + S.grid_off + (long long)iy * K2 + iz;
        const float wb = pick4(w1, b), db = pick4(d1, b), wc = pick4(w2, c), dc = pick4(d2, c);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float v = __ldg(g + (long long)wrapk(f0 - a, K0) * K1 * K2);
            gxs = fmaf(d0[a] * wb * wc, v, gxs);
            gys = fmaf(w0[a] * db * wc, v, gys);
            gzs = fmaf(w0[a] * wb * dc, v, gzs);
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        gxs += __shfl_xor_sync(0xffffffffu, gxs, o);
        gys += __shfl_xor_sync(0xffffffffu, gys, o);
        gzs += __shfl_xor_sync(0xffffffffu, gzs, o);
    }
    if (!valid || sub != 0) return;
    float fx = -q * k0l * gxs, fy = -q * k1l * gys, fz = -q * k2l * gzs;
    if (mode == 0) {
        if (!pme) return;
        // added atomically: the pair kernel adds its part concurrently
        const int k = slot_of ? slot_of[ii] : ii;
        red_add(ffix + k, to_fix(fx, scale, flags + 1));
        red_add(ffix + (size_t)N + k, to_fix(fy, scale, flags + 1));
        red_add(ffix + 2 * (size_t)N + k, to_fix(fz, scale, flags + 1));
    } else {
        int o = perm[ii];
        f_out[3 * (size_t)o] = fx;
        f_out[3 * (size_t)o + 1] = fy;
        f_out[3 * (size_t)o + 2] = fz;
    }
}

// Mesh starts are padded to 64 elements (256 B for float, 512 B for float2) so that
// every batched cuFFT transform sees aligned input and output.
static long long mesh_stride(long long n) { return (n + 63) / 64 * 64; }

cudaError_t pme_setup(nb_handle* h) {
    // Group PME systems by mesh shape; meshes of a group sit at a fixed stride.
    h->fft.clear();
    std::vector<int> order;
    for (int s = 0; s < h->n_sys; ++s)
        if (h->sys_h[s].pme) order.push_back(s);
    long long goff = 0, coff = 0;
    std::vector<bool> done(h->n_sys, false);
    for (size_t a = 0; a < order.size(); ++a) {
        int s = order[a];
        if (done[s]) continue;
        FftGroup g;
        for (int d = 0; d < 3; ++d) g.K[d] = h->sys_h[s].K[d];
        g.count = 0;
        g.grid_off = goff;
        g.cgrid_off = coff;
        long long nr = mesh_stride((long long)g.K[0] * g.K[1] * g.K[2]);
        long long nc = mesh_stride((long long)g.K[0] * g.K[1] * (g.K[2] / 2 + 1));
        g.dist_r = nr;
        g.dist_c = nc;
        for (size_t b = a; b < order.size(); ++b) {
            int t = order[b];
            const SysDev& T = h->sys_h[t];
            if (!done[t] && T.K[0] == g.K[0] && T.K[1] == g.K[1] && T.K[2] == g.K[2]) {
                done[t] = true;
                h->sys_h[t].grid_off = goff;
                h->sys_h[t].cgrid_off = coff;
                goff += nr;
                coff += nc;
                g.count++;
            }
        }
        h->fft.push_back(g);
    }
    h->grid_total = goff;
    h->cgrid_total = coff;
    h->has_pme = goff > 0;
    if (!h->has_pme) return cudaSuccess;
    // convolve block map
    std::vector<int> blk_sys, blk_off(h->n_sys + 1, 0);
    for (int s = 0; s < h->n_sys; ++s) {
        blk_off[s] = (int)blk_sys.size();
        const SysDev& S = h->sys_h[s];
        if (!S.pme) continue;
        long long nc = (long long)S.K[0] * S.K[1] * (S.K[2] / 2 + 1);
        int nb = cdiv(nc, kConvTile);
        for (int b = 0; b < nb; ++b) blk_sys.push_back(s);
    }
    blk_off[h->n_sys] = (int)blk_sys.size();
    h->n_conv_blocks = (int)blk_sys.size();
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) h->allocs.push_back(*p);
        return e;
    };
    cudaError_t e;
    if ((e = alloc((void**)&h->gfix, sizeof(long long) * goff)) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->grid, sizeof(float) * goff)) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->grid2, sizeof(float) * goff)) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->lam_max, sizeof(unsigned))) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->cgrid, sizeof(float2) * coff)) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->green, sizeof(float) * coff)) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->conv_blk_sys, sizeof(int) * blk_sys.size())) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->conv_blk_off, sizeof(int) * blk_off.size())) != cudaSuccess) return e;
    if ((e = alloc((void**)&h->e_pme_blk, sizeof(double) * blk_sys.size())) != cudaSuccess) return e;
    h->kl_max = 0.f;
    for (int s = 0; s < h->n_sys; ++s)
        if (h->sys_h[s].pme)
            for (int d = 0; d < 3; ++d) h->kl_max = std::max(h->kl_max, h->sys_h[s].kl_hi[d]);
    cudaMemset(h->gfix, 0, sizeof(long long) * goff);
    cudaMemset(h->grid, 0, sizeof(float) * goff);
    cudaMemset(h->green, 0, sizeof(float) * coff);
    cudaMemcpy(h->conv_blk_sys, blk_sys.data(), sizeof(int) * blk_sys.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(h->conv_blk_off, blk_off.data(), sizeof(int) * blk_off.size(), cudaMemcpyHostToDevice);
    for (int s = 0; s < h->n_sys; ++s) {
        const SysDev& S = h->sys_h[s];
        if (!S.pme) continue;
        long long nc = (long long)S.K[0] * S.K[1] * (S.K[2] / 2 + 1);
        k_green<<<cdiv(nc, 256), 256>>>(S.K[0], S.K[1], S.K[2], h->desc[s].box[0], h->desc[s].box[1],
                                        h->desc[s].box[2], h->desc[s].alpha, h->desc[s].ke,
                                        h->green + S.cgrid_off);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (auto& g : h->fft) {
        int n[3] = {g.K[0], g.K[1], g.K[2]};
        int nce[3] = {g.K[0], g.K[1], g.K[2] / 2 + 1};
        int dr = (int)g.dist_r, dc = (int)g.dist_c;
        if (cufftPlanMany(&g.r2c, 3, n, n, 1, dr, nce, 1, dc, CUFFT_R2C, g.count) != CUFFT_SUCCESS)
            return cudaErrorUnknown;
        g.has_r2c = true;
        if (cufftPlanMany(&g.c2r, 3, n, nce, 1, dc, n, 1, dr, CUFFT_C2R, g.count) != CUFFT_SUCCESS)
            return cudaErrorUnknown;
        g.has_c2r = true;
    }
    return cudaDeviceSynchronize();
}

static void spread(nb_handle* h, const float4* x, cudaStream_t st) {
    int N = h->n_atoms;
    k_spread<<<cdiv((long long)N * 16, 256), 256, 0, st>>>(N, x, h->sid, h->sys, h->gfix, (float)h->gscale);
    launch_pdl(k_grid_convert, cdiv(h->grid_total, 256), 256, 0, st, h->grid_total, h->gfix, h->grid, 1.0 / h->gscale);
}

void launch_pme_spread(nb_handle* h, const float4* x, cudaStream_t st) { spread(h, x, st); }

static int fft_on(nb_handle* h, float* mesh, int inverse, cudaStream_t st) {
    for (auto& g : h->fft) {
        if (!inverse) {
            cufftSetStream(g.r2c, st);
            if (cufftExecR2C(g.r2c, mesh + g.grid_off, reinterpret_cast<cufftComplex*>(h->cgrid + g.cgrid_off)) !=
                CUFFT_SUCCESS)
                return 1;
        } else {
            cufftSetStream(g.c2r, st);
            if (cufftExecC2R(g.c2r, reinterpret_cast<cufftComplex*>(h->cgrid + g.cgrid_off), mesh + g.grid_off) !=
                CUFFT_SUCCESS)
                return 1;
        }
    }
    return 0;
}

int launch_pme_fft(nb_handle* h, int inverse, cudaStream_t st) { return fft_on(h, h->grid, inverse, st); }

void launch_pme_convolve(nb_handle* h, cudaStream_t st) {
    launch_pdl(k_convolve, h->n_conv_blocks, kConvThreads, 0, st, h->conv_blk_sys, h->conv_blk_off, h->sys, h->cgrid,
                                                          h->green, h->e_pme_blk);
}

void launch_pme_gather(nb_handle* h, const float4* x, const int* slot_of, cudaStream_t st) {
    int N = h->n_atoms;
    k_gather<<<cdiv((long long)N * 16, 256), 256, 0, st>>>(N, x, h->sid, h->sys, h->grid, h->ffix, nullptr,
                                                           h->perm, slot_of, h->fscale, 0, h->flags);
}

// ---------------------------------------------------------------- reciprocal-space VJP
// With F_i = -q_i sum_k grad theta_i(k) phi(k) and phi = C Q (C the symmetric convolution
// with G), lam . F = -<psi, phi> where psi(k) = sum_i q_i lam_i . grad theta_i(k).  Then
//   d(lam . F)/dx_j = -q_j sum_k (Hess theta_j(k) lam_j) phi(k) - q_j sum_k grad theta_j(k) chi(k)
//   d(lam . F)/dq_j = -sum_k (lam_j . grad theta_j(k)) phi(k) - sum_k theta_j(k) chi(k)
// with chi = C psi: psi is spread like Q (int64 fixed point, scale 2^32 over the largest
// |lam| K/L, a power of two), convolved on a second mesh, and both meshes are gathered.

// Second derivatives of the order-4 pieces (u units): the cubic weights differentiated twice.
__device__ __forceinline__ void bspline4_d2(float t, float d2[4]) {
    d2[0] = t;
    d2[1] = 1.f - 3.f * t;
    d2[2] = 3.f * t - 2.f;
    d2[3] = 1.f - t;
}

__global__ void k_absmax(int N, const float4* __restrict__ lam, unsigned* __restrict__ out) {
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float4 l = lam[i];
        m = fmaxf(m, fmaxf(fabsf(l.x), fmaxf(fabsf(l.y), fabsf(l.z))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

// 2^32 over the largest |lam| K/L, rounded down to a power of two (so the round trip of
// the fixed-point mesh is exact in its scale).
__device__ __forceinline__ float psi_scale(const unsigned* lam_max, float kl_max) {
    const float m = fmaxf(__uint_as_float(*lam_max) * kl_max, 1e-30f);
    return ldexpf(1.f, 31 - ilogbf(m));
}

__global__ void k_spread_vjp(int N, const float4* __restrict__ xs, const float4* __restrict__ lam,
                             const int* __restrict__ sid, const SysDev* __restrict__ sys,
                             long long* __restrict__ gfix, const unsigned* __restrict__ lam_max, float kl_max) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt >> 4, sub = gt & 15;
    if (i >= N) return;
    const SysDev& S = sys[sid[i]];
    if (!S.pme) return;
    const float vs = psi_scale(lam_max, kl_max);
    const float4 p = xs[i];
    const float4 l = lam[i];
    int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
    int f0, f1, f2;
    float t0, t1, t2;
    frac_coord(p.x, K0, S.kl_hi[0], S.kl_lo[0], f0, t0);
    frac_coord(p.y, K1, S.kl_hi[1], S.kl_lo[1], f1, t1);
    frac_coord(p.z, K2, S.kl_hi[2], S.kl_lo[2], f2, t2);
    float w0[4], w1[4], w2[4], d0[4], d1[4], d2[4];
    bspline4(t0, w0, d0);
    bspline4(t1, w1, d1);
    bspline4(t2, w2, d2);
    const float lu0 = l.x * S.kl_hi[0], lu1 = l.y * S.kl_hi[1], lu2 = l.z * S.kl_hi[2];  // lam in u units
    int a = sub >> 2, b = sub & 3;
    int ix = wrapk(f0 - a, K0), iy = wrapk(f1 - b, K1);
    long long* g = gfix + S.grid_off + ((long long)ix * K1 + iy) * K2;
    const float wa = pick4(w0, a), da = pick4(d0, a), wb = pick4(w1, b), db = pick4(d1, b);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float wv = lu0 * da * wb * w2[c] + lu1 * wa * db * w2[c] + lu2 * wa * wb * d2[c];
        red_add(g + wrapk(f2 - c, K2), __float2ll_rn(p.w * wv * vs));
    }
}

__global__ void k_grid_convert_dyn(long long n, long long* __restrict__ gfix, float* __restrict__ grid,
                                   const unsigned* __restrict__ lam_max, float kl_max) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double inv = 1.0 / (double)psi_scale(lam_max, kl_max);
    grid[k] = (float)((double)gfix[k] * inv);
    gfix[k] = 0;
}

// 16 lanes per atom as in k_gather; adds (gx, gq) to the slot-order VJP output.
__global__ void k_gather_vjp(int N, const float4* __restrict__ xs, const float4* __restrict__ lam,
                             const int* __restrict__ sid, const SysDev* __restrict__ sys,
                             const float* __restrict__ phi, const float* __restrict__ chi,
                             float4* __restrict__ gx_s) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt >> 4, sub = gt & 15;
    bool valid = i < N;
    int ii = valid ? i : N - 1;
    const SysDev& S = sys[sid[ii]];
    bool pme = valid && S.pme;
    float A[3] = {0.f, 0.f, 0.f}, B[3] = {0.f, 0.f, 0.f}, c1 = 0.f, c2 = 0.f;
    float q = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f;
    if (pme) {
        const float4 p = xs[ii];
        const float4 l = lam[ii];
        q = p.w;
        s0 = S.kl_hi[0];
        s1 = S.kl_hi[1];
        s2 = S.kl_hi[2];
        int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
        int f0, f1, f2;
        float t0, t1, t2;
        frac_coord(p.x, K0, S.kl_hi[0], S.kl_lo[0], f0, t0);
        frac_coord(p.y, K1, S.kl_hi[1], S.kl_lo[1], f1, t1);
        frac_coord(p.z, K2, S.kl_hi[2], S.kl_lo[2], f2, t2);
        float w0[4], w1[4], w2[4], d0[4], d1[4], d2[4], e0[4], e1[4], e2[4];
        bspline4(t0, w0, d0);
        bspline4(t1, w1, d1);
        bspline4(t2, w2, d2);
        bspline4_d2(t0, e0);
        bspline4_d2(t1, e1);
        bspline4_d2(t2, e2);
        const float lu0 = l.x * s0, lu1 = l.y * s1, lu2 = l.z * s2;
        int a = sub >> 2, b = sub & 3;
        int ix = wrapk(f0 - a, K0), iy = wrapk(f1 - b, K1);
        const long long row = S.grid_off + ((long long)ix * K1 + iy) * K2;
        const float wa = pick4(w0, a), da = pick4(d0, a), ea = pick4(e0, a);
        const float wb = pick4(w1, b), db = pick4(d1, b), eb = pick4(e1, b);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long k = row + wrapk(f2 - c, K2);
            const float pv = __ldg(phi + k), hv = __ldg(chi + k);
            const float th = wa * wb * w2[c];
            const float g0 = da * wb * w2[c], g1 = wa * db * w2[c], g2 = wa * wb * d2[c];
            const float h01 = da * db * w2[c], h02 = da * wb * d2[c], h12 = wa * db * d2[c];
            const float hx = ea * wb * w2[c] * lu0 + h01 * lu1 + h02 * lu2;
            const float hy = h01 * lu0 + wa * eb * w2[c] * lu1 + h12 * lu2;
            const float hz = h02 * lu0 + h12 * lu1 + wa * wb * e2[c] * lu2;
            A[0] = fmaf(hx, pv, A[0]);
            A[1] = fmaf(hy, pv, A[1]);
            A[2] = fmaf(hz, pv, A[2]);
            B[0] = fmaf(g0, hv, B[0]);
            B[1] = fmaf(g1, hv, B[1]);
            B[2] = fmaf(g2, hv, B[2]);
            c1 = fmaf(lu0 * g0 + lu1 * g1 + lu2 * g2, pv, c1);
            c2 = fmaf(th, hv, c2);
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            A[d] += __shfl_xor_sync(0xffffffffu, A[d], o);
            B[d] += __shfl_xor_sync(0xffffffffu, B[d], o);
        }
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    if (!pme || sub != 0) return;
    float4 g = gx_s[ii];
    g.x -= q * s0 * (A[0] + B[0]);
    g.y -= q * s1 * (A[1] + B[1]);
    g.z -= q * s2 * (A[2] + B[2]);
    g.w -= c1 + c2;
    gx_s[ii] = g;
}

int launch_pme_vjp(nb_handle* h, cudaStream_t st) {
    if (!h->has_pme) return 0;
    int N = h->n_atoms;
    // forward: phi on the first mesh, the reciprocal energy and forces (added to ffix)
    if (launch_pme(h, st)) return 1;
    // psi on the second mesh, chi = C psi
    cudaMemsetAsync(h->lam_max, 0, sizeof(unsigned), st);
    k_absmax<<<std::min(cdiv(N, 256), 1184), 256, 0, st>>>(N, h->lam, h->lam_max);
    k_spread_vjp<<<cdiv((long long)N * 16, 256), 256, 0, st>>>(N, h->xs, h->lam, h->sid, h->sys, h->gfix,
                                                                h->lam_max, h->kl_max);
    k_grid_convert_dyn<<<cdiv(h->grid_total, 256), 256, 0, st>>>(h->grid_total, h->gfix, h->grid2, h->lam_max,
                                                                 h->kl_max);
    if (fft_on(h, h->grid2, 0, st)) return 1;
    launch_pdl(k_convolve, h->n_conv_blocks, kConvThreads, 0, st, h->conv_blk_sys, h->conv_blk_off, h->sys, h->cgrid,
                                                          h->green, nullptr);
    if (fft_on(h, h->grid2, 1, st)) return 1;
    k_gather_vjp<<<cdiv((long long)N * 16, 256), 256, 0, st>>>(N, h->xs, h->lam, h->sid, h->sys, h->grid,
                                                                h->grid2, h->gx_s);
    return 0;
}

int launch_pme(nb_handle* h, cudaStream_t st) {
    if (!h->has_pme) return 0;
    launch_pme_spread(h, h->xs, st);
    if (launch_pme_fft(h, 0, st)) return 1;
    launch_pme_convolve(h, st);
    if (launch_pme_fft(h, 1, st)) return 1;
    launch_pme_gather(h, h->xs, nullptr, st);
    return 0;
}

void launch_pme_spread_only(nb_handle* h, float* grid_out, cudaStream_t st) {
    if (!h->has_pme) return;
    spread(h, h->xs, st);
    long long off = 0;
    for (int s = 0; s < h->n_sys; ++s) {
        const SysDev& S = h->sys_h[s];
        if (!S.pme) continue;
        long long nr = (long long)S.K[0] * S.K[1] * S.K[2];
        cudaMemcpyAsync(grid_out + off, h->grid + S.grid_off, sizeof(float) * nr, cudaMemcpyDeviceToDevice, st);
        off += nr;
    }
}

void launch_pme_gather_only(nb_handle* h, const float* phi, float* f_out, cudaStream_t st) {
    int N = h->n_atoms;
    cudaMemsetAsync(f_out, 0, sizeof(float) * 3 * (size_t)N, st);
    if (!h->has_pme) return;
    long long off = 0;
    for (int s = 0; s < h->n_sys; ++s) {
        const SysDev& S = h->sys_h[s];
        if (!S.pme) continue;
        long long nr = (long long)S.K[0] * S.K[1] * S.K[2];
        cudaMemcpyAsync(h->grid + S.grid_off, phi + off, sizeof(float) * nr, cudaMemcpyDeviceToDevice, st);
        off += nr;
    }
    k_gather<<<cdiv((long long)N * 16, 256), 256, 0, st>>>(N, h->xs, h->sid, h->sys, h->grid, nullptr, f_out,
                                                           h->perm, nullptr, h->fscale, 1, h->flags);
}

}  // namespace nb

// ------------------------------------------------------------------------------
// pme_spread_static: the charge spreading above for callers that cannot allocate
// device memory.  Its int64 accumulation mesh is a file-scope device array of
// NB_STATIC_MESH_MAX points that every GPU loading the library keeps until exit;
// host code reaches it only through the address cudaGetSymbolAddress returns (in
// host code the array's name is a stand-in, not a device address).

namespace nb {
namespace {

static __device__ __align__(256) long long g_static_mesh[NB_STATIC_MESH_MAX];

// Device address of g_static_mesh in the current context.  It is looked up on every call
// (the lookup allocates nothing): an address kept from an earlier call would be stale after
// cudaDeviceReset or once a new primary context is created on the device.
cudaError_t static_mesh_address(long long** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_mesh);
    if (e != cudaSuccess) return e;
    *out = static_cast<long long*>(p);
    return cudaSuccess;
}

// Same arithmetic as k_spread, reading caller-order positions and wrapping them itself.
__global__ void k_spread_static(int N, const float4* __restrict__ xq, float L0, float L1, float L2, float iL0,
                                float iL1, float iL2, int K0, int K1, int K2, float kh0, float kh1, float kh2,
                                float kl0, float kl1, float kl2, long long* __restrict__ mesh, float gscale) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt >> 4, sub = gt & 15;
    if (i >= N) return;
    float4 p = xq[i];
    p.x = wrap1(p.x, L0, iL0);
    p.y = wrap1(p.y, L1, iL1);
    p.z = wrap1(p.z, L2, iL2);
    int f0, f1, f2;
    float t0, t1, t2;
    frac_coord(p.x, K0, kh0, kl0, f0, t0);
    frac_coord(p.y, K1, kh1, kl1, f1, t1);
    frac_coord(p.z, K2, kh2, kl2, f2, t2);
    float w0[4], w1[4], w2[4], d[4];
    bspline4(t0, w0, d);
    bspline4(t1, w1, d);
    bspline4(t2, w2, d);
    int a = sub >> 2, b = sub & 3;
    int ix = wrapk(f0 - a, K0), iy = wrapk(f1 - b, K1);
    float wxy = p.w * w0[a] * w1[b];
    long long* g = mesh + ((long long)ix * K1 + iy) * K2;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int iz = wrapk(f2 - c, K2);
        red_add(g + iz, __float2ll_rn(wxy * w2[c] * gscale));
    }
}

__global__ void k_static_mesh_out(long long n, const long long* __restrict__ mesh, float* __restrict__ grid,
                                  double ginv) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    grid[k] = (float)((double)mesh[k] * ginv);
}

}  // namespace
}  // namespace nb

extern "C" nb_status pme_spread_static(const float* xq, int32_t n_atoms, const double* box, const int32_t* mesh,
                                       float* grid, void* stream) {
    using namespace nb;
    // an empty system reads no positions: xq may then be NULL (its mesh is all zeros)
    if ((!xq && n_atoms > 0) || !grid || !box || !mesh || n_atoms < 0) return NB_ERR_ARG;
    // each factor is checked against the capacity before it is multiplied in, so the
    // product cannot wrap (three sizes up to 2^31 would overflow 64 bits)
    long long npts = 1;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0.0) || !std::isfinite(box[d]) || mesh[d] < 4 || mesh[d] > NB_STATIC_MESH_MAX) return NB_ERR_ARG;
        npts *= mesh[d];
        if (npts > NB_STATIC_MESH_MAX) return NB_ERR_ARG;
    }
    long long* scratch = nullptr;
    if (static_mesh_address(&scratch) != cudaSuccess) return NB_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the mesh keeps the previous call's sums: clear the part this call uses
    if (cudaMemsetAsync(scratch, 0, sizeof(long long) * (size_t)npts, st) != cudaSuccess) return NB_ERR_CUDA;
    float kh[3], kl[3];
    for (int d = 0; d < 3; ++d) {
        double r = mesh[d] / box[d];
        kh[d] = (float)r;
        kl[d] = (float)(r - (double)kh[d]);
    }
    const double gscale = std::ldexp(1.0, 32);
    if (n_atoms > 0)
        k_spread_static<<<cdiv((long long)n_atoms * 16, 256), 256, 0, st>>>(
            n_atoms, reinterpret_cast<const float4*>(xq), (float)box[0], (float)box[1], (float)box[2],
            (float)(1.0 / box[0]), (float)(1.0 / box[1]), (float)(1.0 / box[2]), mesh[0], mesh[1], mesh[2], kh[0],
            kh[1], kh[2], kl[0], kl[1], kl[2], scratch, (float)gscale);
    k_static_mesh_out<<<cdiv(npts, 256), 256, 0, st>>>(npts, scratch, grid, 1.0 / gscale);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
