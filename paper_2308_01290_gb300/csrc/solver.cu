// Algorithm 1 of Sec. II-D on the GPU.
//
// Maps live in batch pools (one pool per field, slices at SliceGeom::off,
// rows of `pitch` elements).  One iteration is:
//   k_thr_rhs   eq. sol_hv for f1, f2, rho_e, z (periodic forward differences,
//               hard threshold at lambda/beta, tie -> 0) and the right-hand
//               sides of the f1 / f2 closed forms; beta~ div(h, v) of rho_e, z
//   FFT solve   f = F^-1[F(rhs) / (c_f + beta K)], K = |F dx|^2 + |F dy|^2
//   k_synth     mu(E_j) from the new f (eq. mac_E1/E2), rhs of the rho_e
//               update and the Z^m normal equations (a^2, a b + beta~ div)
//   FFT solve   rho_e = F^-1[F(rhs) / (1 + beta~ K)]
//   PCG         [diag(a^2) + beta~ L] z = rhs, warm start, preconditioner
//               D^-1/2 (mean(a^2) + beta~ L)^-1 D^-1/2 with D = diag(a^2+4beta~)
//               normalised to 1 at mean(a^2)
//   k_next_beta beta <- kappa beta, beta~ = tau beta
// Sums for reductions are FP64 in a fixed order (deterministic).
#include <cmath>
#include <cstdio>
#include <vector>

#include "ctx.h"
#include "fft.cuh"

namespace recon {

template <typename T>
struct Ptrs {
    T* f[kNumFields];
    cplx<T>* s[kNumSpectra];
    unsigned long long* acct;   // algorithmic bytes per kernel family
};

// Adds the algorithmic bytes of one processed item to its family's counter.
__device__ __forceinline__ void account(unsigned long long* acct, int fam, long long bytes) {
    if (threadIdx.x == 0) atomicAdd(acct + fam, (unsigned long long)bytes);
}

__device__ __forceinline__ long long tile_px(const SliceGeom& g, const Item& it) {
    const int w = g.nx - it.a < kTile ? g.nx - it.a : kTile;
    const int h = g.ny - it.b < kTile ? g.ny - it.b : kTile;
    return (long long)w * h;
}

struct FftJobs {
    int n;
    int in[3], spec[3], out[3], coef[3];
};

// --------------------------------------------------------------------------
// helpers
// --------------------------------------------------------------------------

__device__ __forceinline__ bool keep_grad(float dx, float dy, float thr) {
    // (dx)^2 + (dy)^2 > lambda/beta, each operation rounded (no contraction)
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) > thr;
}
__device__ __forceinline__ bool keep_grad(double dx, double dy, double thr) {
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) > thr;
}
template <typename T>
__device__ __forceinline__ T sub_rn(T a, T b);
template <>
__device__ __forceinline__ float sub_rn<float>(float a, float b) { return __fsub_rn(a, b); }
template <>
__device__ __forceinline__ double sub_rn<double>(double a, double b) { return __dsub_rn(a, b); }

template <typename T>
__device__ __forceinline__ T thr_of(const SliceState& st);
template <>
__device__ __forceinline__ float thr_of<float>(const SliceState& st) { return st.thr_f; }
template <>
__device__ __forceinline__ double thr_of<double>(const SliceState& st) { return st.thr_d; }

// --------------------------------------------------------------------------
// input load and initialisation (Alg. 1, Initialization)
// --------------------------------------------------------------------------

template <typename T>
__global__ void k_load(ItemList L, const SliceGeom* G, const SliceConst* C, const float* __restrict__ lo,
                       const float* __restrict__ hi, T* muL, T* muH) {
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceGeom g = G[it.slice];
        const double s = C[it.slice].inv_S;
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int x = it.a + (q & (kTile - 1)), y = it.b + q / kTile;
            if (x >= g.nx || y >= g.ny) continue;
            const long long e = g.ext_off + (long long)y * g.nx + x;
            const long long d = g.off + (long long)y * g.pitch + x;
            muL[d] = T((double)lo[e] * s);
            muH[d] = T((double)hi[e] * s);
        }
    }
}

template <typename T>
__global__ void k_init(ItemList L, const SliceGeom* G, const SliceConst* C, Ptrs<T> P) {
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceGeom g = G[it.slice];
        const SliceConst c = C[it.slice];
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int x = it.a + (q & (kTile - 1)), y = it.b + q / kTile;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const double uL = P.f[RECON_F_MUL][d], uH = P.f[RECON_F_MUH][d];
            // Cramer on eq. lac_EL / lac_EH
            const double f1 = (c.a11 * uL - c.a10 * uH) / c.det;
            const double f2 = (c.a00 * uH - c.a01 * uL) / c.det;
            // eq. mac_E1 / mac_E2
            const double m1 = c.b00 * f1 + c.b10 * f2;
            const double m2 = c.b01 * f1 + c.b11 * f2;
            // eq. rho_e, eq. Z_m (normalised)
            const double rho = (m1 * c.r - m2) / c.c_rho;
            const double a = (m1 * c.P2 - m2 * c.P1) / c.a_w;
            const double b = (m2 * c.psi1 - m1 * c.psi2) / c.a_w;
            double z = 1.0;
            if (a != 0.0 && rho >= c.rho_air) z = fmin(fmax(b / a, 0.0), c.zclip_hi);
            P.f[RECON_F_F1][d] = T(f1);
            P.f[RECON_F_F2][d] = T(f2);
            P.f[RECON_F_RHO][d] = T(rho);
            P.f[RECON_F_Z][d] = T(z);
        }
    }
}

// --------------------------------------------------------------------------
// K1: hard threshold (eq. sol_hv) + right-hand sides
// --------------------------------------------------------------------------

template <typename T, bool STATS>
__global__ void __launch_bounds__(kStencilThreads) k_thr_rhs(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                             SliceState* S, Ptrs<T> P) {
    __shared__ T sm[4][kTile + 2][kTile + 2];
    __shared__ double red[9 * 32];
    const int maps[4] = {RECON_F_F1, RECON_F_F2, RECON_F_RHO, RECON_F_Z};
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState st = S[it.slice];
        if (!st.active) continue;
        const SliceGeom g = G[it.slice];
        const SliceConst c = C[it.slice];
        account(P.acct, KF_THR_RHS, tile_px(g, it) * 10 * (long long)sizeof(T));
        for (int q = threadIdx.x; q < (kTile + 2) * (kTile + 2); q += blockDim.x) {
            const int ly = q / (kTile + 2), lx = q - ly * (kTile + 2);
            const int gy = wrap(it.b - 1 + ly, g.ny), gx = wrap(it.a - 1 + lx, g.nx);
            const long long d = g.off + (long long)gy * g.pitch + gx;
#pragma unroll
            for (int m = 0; m < 4; ++m) sm[m][ly][lx] = P.f[maps[m]][d];
        }
        __syncthreads();
        const T thr = thr_of<T>(st);
        const T beta = T(st.beta), beta_t = T(st.beta_t);
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int lx = q & (kTile - 1), ly = q / kTile;
            const int x = it.a + lx, y = it.b + ly;
            if (x >= g.nx || y >= g.ny) continue;
            T div[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const T gc = sm[m][ly + 1][lx + 1];
                const T dx = sub_rn(sm[m][ly + 1][lx + 2], gc);
                const T dy = sub_rn(sm[m][ly + 2][lx + 1], gc);
                const T dxl = sub_rn(gc, sm[m][ly + 1][lx]);
                const T dyl = sub_rn(sm[m][ly + 2][lx], sm[m][ly + 1][lx]);
                const T dxu = sub_rn(sm[m][ly][lx + 2], sm[m][ly][lx + 1]);
                const T dyu = sub_rn(gc, sm[m][ly][lx + 1]);
                const bool k0 = keep_grad(dx, dy, thr);
                const bool kl = keep_grad(dxl, dyl, thr);
                const bool ku = keep_grad(dxu, dyu, thr);
                const T h0 = k0 ? dx : T(0), v0 = k0 ? dy : T(0);
                const T hl = kl ? dxl : T(0), vu = ku ? dyu : T(0);
                div[m] = (hl - h0) + (vu - v0);
                if (STATS) {
                    if (!k0) acc[4] += (double)dx * dx + (double)dy * dy;
                    acc[5 + m] += k0 ? 1.0 : 0.0;
                }
            }
            const long long d = g.off + (long long)y * g.pitch + x;
            const T f1 = sm[0][ly + 1][lx + 1], f2 = sm[1][ly + 1][lx + 1];
            const T rho = sm[2][ly + 1][lx + 1], z = sm[3][ly + 1][lx + 1];
            const T uL = P.f[RECON_F_MUL][d], uH = P.f[RECON_F_MUH][d];
            const T M1 = rho * (T(c.P1) * z + T(c.psi1));
            const T M2 = rho * (T(c.P2) * z + T(c.psi2));
            const T base1 = T(c.a00) * uL + T(c.a01) * uH + T(c.b00) * M1 + T(c.b01) * M2;
            const T base2 = T(c.a10) * uL + T(c.a11) * uH + T(c.b10) * M1 + T(c.b11) * M2;
            P.f[RECON_F_RHS_F1][d] = base1 - T(c.c12) * f2 + beta * div[0];
            P.f[RECON_F_RHS_F2][d] = (c.order ? base2 : base2 - T(c.c12) * f1) + beta * div[1];
            P.f[RECON_F_DIV_RHO][d] = beta_t * div[2];
            P.f[RECON_F_DIV_Z][d] = beta_t * div[3];
            if (STATS) {
                const double dL = c.a00 * (double)f1 + c.a10 * (double)f2 - (double)uL;
                const double dH = c.a01 * (double)f1 + c.a11 * (double)f2 - (double)uH;
                const double m1 = c.b00 * (double)f1 + c.b10 * (double)f2;
                const double m2 = c.b01 * (double)f1 + c.b11 * (double)f2;
                const double e1 = (double)rho * (c.P1 * (double)z + c.psi1) - m1;
                const double e2 = (double)rho * (c.P2 * (double)z + c.psi2) - m2;
                acc[0] += dL * dL;
                acc[1] += dH * dH;
                acc[2] += e1 * e1;
                acc[3] += e2 * e2;
            }
        }
        if (STATS) {
            block_sum<9>(acc, red);
            double tot[9];
            if (item_reduce<9>(L, w, it.slice, acc, tot)) {
                SliceState& so = S[it.slice];
                for (int q = 0; q < 5; ++q) so.stat[q] = tot[q];
                for (int m = 0; m < 4; ++m) so.nnz[m] = (long long)(tot[5 + m] + 0.5);
            }
        }
        __syncthreads();
    }
}

// Gauss-Seidel variant: f2's right-hand side takes the new f1.
template <typename T>
__global__ void k_gs_fix(ItemList L, const SliceGeom* G, const SliceConst* C, const SliceState* S, Ptrs<T> P) {
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        if (!S[it.slice].active) continue;
        const SliceGeom g = G[it.slice];
        const T c12 = T(C[it.slice].c12);
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int x = it.a + (q & (kTile - 1)), y = it.b + q / kTile;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            P.f[RECON_F_RHS_F2][d] -= c12 * P.f[RECON_F_F1][d];
        }
    }
}

// --------------------------------------------------------------------------
// FFT-diagonalised solve: rows (R2C, two real rows per complex FFT),
// columns (FFT, divide by c + beta K, inverse FFT), rows (C2R).
// --------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void solve_coef(int kind, const SliceConst& c, const SliceState& st, double& cc,
                                           double& bb) {
    switch (kind) {
        case 0: cc = c.c_f1; bb = st.beta; break;
        case 1: cc = c.c_f2; bb = st.beta; break;
        case 2: cc = 1.0; bb = st.beta_t; break;
        default: cc = st.abar2; bb = st.beta_t; break;
    }
}

__device__ __forceinline__ bool job_skip(const SliceState& st, int kind) {
    return !st.active || (kind == 3 && st.cg_done);
}

// MODE 0: input is a field.  MODE 1: input is D^-1/2-scaled CG residual.
template <typename T, int MODE>
__global__ void __launch_bounds__(kFftThreads) k_rows_fwd(ItemList L, const SliceGeom* G, const SliceState* S,
                                                           Ptrs<T> P, FftJobs J, int buf_elems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* bufB = bufA + buf_elems;
    cplx<T>* tw = bufB + buf_elems;
    const int total = L.n_items * J.n;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int job = w / L.n_items, item = w - job * L.n_items;
        const Item it = L.items[item];
        const SliceState st = S[it.slice];
        if (job_skip(st, J.coef[job])) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.nx, pair0 = it.a, np = it.b;
        {
            const int rows = (g.ny - 2 * pair0 < 2 * np) ? g.ny - 2 * pair0 : 2 * np;
            account(P.acct, MODE ? KF_ROWS_FWD_PRE : KF_ROWS_FWD,
                    (long long)rows * ((MODE ? 2 : 1) * N * (long long)sizeof(T) + g.nh * 2 * (long long)sizeof(T)));
        }
        fill_twiddles(tw, N);
        const T* in = P.f[J.in[job]];
        const T* a2 = P.f[RECON_F_A2];
        const T num = T(st.abar2 + 4.0 * st.beta_t), b4 = T(4.0 * st.beta_t);
        for (int q = threadIdx.x; q < np * N; q += blockDim.x) {
            const int b = q / N, n = q - b * N;
            const int row = 2 * (pair0 + b);
            const long long d0 = g.off + (long long)row * g.pitch + n;
            T v0 = in[d0], v1 = T(0);
            const bool has1 = row + 1 < g.ny;
            if (has1) v1 = in[d0 + g.pitch];
            if (MODE == 1) {
                v0 *= sqrt(num / (a2[d0] + b4));
                if (has1) v1 *= sqrt(num / (a2[d0 + g.pitch] + b4));
            }
            bufA[b * N + n] = {v0, v1};
        }
        __syncthreads();
        const cplx<T>* res = fft_batch<T>(bufA, bufB, N, np, N, tw, -1);
        cplx<T>* sp = P.s[J.spec[job]];
        for (int q = threadIdx.x; q < np * g.nh; q += blockDim.x) {
            const int b = q / g.nh, k = q - b * g.nh;
            const int row = 2 * (pair0 + b);
            const cplx<T> zk = res[b * N + k];
            const cplx<T> zc = res[b * N + (k == 0 ? 0 : N - k)];
            // A = (Z_k + conj Z_-k)/2, B = (Z_k - conj Z_-k)/(2i)
            const cplx<T> A = {T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
            const cplx<T> B = {T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
            const long long e = g.coff + (long long)row * g.cpitch + k;
            sp[e] = A;
            if (row + 1 < g.ny) sp[e + g.cpitch] = B;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_cols(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                       const SliceState* S, Ptrs<T> P, FftJobs J, int buf_elems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* bufB = bufA + buf_elems;
    cplx<T>* tw = bufB + buf_elems;
    const int total = L.n_items * J.n;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int job = w / L.n_items, item = w - job * L.n_items;
        const Item it = L.items[item];
        const SliceState st = S[it.slice];
        if (job_skip(st, J.coef[job])) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.ny, col0 = it.a, nc = it.b, ld = N + 1;
        account(P.acct, J.coef[job] == 3 ? KF_COLS_PRE : KF_COLS, (long long)nc * N * 4 * (long long)sizeof(T));
        fill_twiddles(tw, N);
        cplx<T>* sp = P.s[J.spec[job]];
        for (int q = threadIdx.x; q < nc * N; q += blockDim.x) {
            const int y = q / nc, cc = q - y * nc;
            bufA[cc * ld + y] = sp[g.coff + (long long)y * g.cpitch + col0 + cc];
        }
        __syncthreads();
        cplx<T>* res = fft_batch<T>(bufA, bufB, N, nc, ld, tw, -1);
        double cst, bet;
        solve_coef<T>(J.coef[job], C[it.slice], st, cst, bet);
        const T inv_n = T(1.0 / ((double)g.nx * (double)g.ny));
        for (int q = threadIdx.x; q < nc * N; q += blockDim.x) {
            const int cc = q / N, ky = q - cc * N;
            T sx = sin(T(M_PI) * T(col0 + cc) / T(g.nx));
            T sy = sin(T(M_PI) * T(ky) / T(N));
            const T den = T(cst) + T(bet) * (T(4) * sx * sx + T(4) * sy * sy);
            const T sc = inv_n / den;
            cplx<T> v = res[cc * ld + ky];
            res[cc * ld + ky] = {v.x * sc, v.y * sc};
        }
        __syncthreads();
        cplx<T>* other = (res == bufA) ? bufB : bufA;
        const cplx<T>* out = fft_batch<T>(res, other, N, nc, ld, tw, +1);
        for (int q = threadIdx.x; q < nc * N; q += blockDim.x) {
            const int y = q / nc, cc = q - y * nc;
            sp[g.coff + (long long)y * g.cpitch + col0 + cc] = out[cc * ld + y];
        }
        __syncthreads();
    }
}

// MODE 0: write the field.  MODE 1: y = D^-1/2 x into CG_Y and reduce r.y.
template <typename T, int MODE>
__global__ void __launch_bounds__(kFftThreads) k_rows_inv(ItemList L, const SliceGeom* G, SliceState* S, Ptrs<T> P,
                                                           FftJobs J, int buf_elems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* bufB = bufA + buf_elems;
    cplx<T>* tw = bufB + buf_elems;
    __shared__ double red[32];
    const int total = L.n_items * J.n;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int job = w / L.n_items, item = w - job * L.n_items;
        const Item it = L.items[item];
        const SliceState st = S[it.slice];
        if (job_skip(st, J.coef[job])) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.nx, pair0 = it.a, np = it.b;
        {
            const int rows = (g.ny - 2 * pair0 < 2 * np) ? g.ny - 2 * pair0 : 2 * np;
            account(P.acct, MODE ? KF_ROWS_INV_PRE : KF_ROWS_INV,
                    (long long)rows * ((MODE ? 3 : 1) * N * (long long)sizeof(T) + g.nh * 2 * (long long)sizeof(T)));
        }
        fill_twiddles(tw, N);
        const cplx<T>* sp = P.s[J.spec[job]];
        for (int q = threadIdx.x; q < np * N; q += blockDim.x) {
            const int b = q / N, n = q - b * N;
            const int row = 2 * (pair0 + b);
            const bool herm = n >= g.nh;
            const int k = herm ? N - n : n;
            const long long e = g.coff + (long long)row * g.cpitch + k;
            cplx<T> A = sp[e], B = {T(0), T(0)};
            if (row + 1 < g.ny) B = sp[e + g.cpitch];
            if (herm) {
                A.y = -A.y;
                B.y = -B.y;
            }
            bufA[b * N + n] = {A.x - B.y, A.y + B.x};
        }
        __syncthreads();
        const cplx<T>* res = fft_batch<T>(bufA, bufB, N, np, N, tw, +1);
        T* out = P.f[J.out[job]];
        double acc[1] = {0.0};
        const T* a2 = P.f[RECON_F_A2];
        const T* r = P.f[RECON_F_CG_R];
        const T num = T(st.abar2 + 4.0 * st.beta_t), b4 = T(4.0 * st.beta_t);
        for (int q = threadIdx.x; q < np * N; q += blockDim.x) {
            const int b = q / N, n = q - b * N;
            const int row = 2 * (pair0 + b);
            const long long d0 = g.off + (long long)row * g.pitch + n;
            const cplx<T> v = res[b * N + n];
            if (MODE == 0) {
                out[d0] = v.x;
                if (row + 1 < g.ny) out[d0 + g.pitch] = v.y;
            } else {
                const T y0 = v.x * sqrt(num / (a2[d0] + b4));
                out[d0] = y0;
                acc[0] += (double)y0 * (double)r[d0];
                if (row + 1 < g.ny) {
                    const long long d1 = d0 + g.pitch;
                    const T y1 = v.y * sqrt(num / (a2[d1] + b4));
                    out[d1] = y1;
                    acc[0] += (double)y1 * (double)r[d1];
                }
            }
        }
        if (MODE == 1) {
            block_sum<1>(acc, red);
            double tot[1];
            if (item_reduce<1>(L, item, it.slice, acc, tot)) {
                SliceState& so = S[it.slice];
                so.betacg = (so.cg_it == 0) ? 0.0 : tot[0] / so.ry;
                so.ry = tot[0];
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// synthesis at E1/E2 from the new f, rho_e rhs, Z^m normal equations
// --------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_synth(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                           SliceState* S, Ptrs<T> P) {
    __shared__ double red[2 * 32];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        if (!S[it.slice].active) continue;
        const SliceGeom g = G[it.slice];
        const SliceConst c = C[it.slice];
        account(P.acct, KF_SYNTH, tile_px(g, it) * 7 * (long long)sizeof(T));
        double acc[2] = {0.0, 0.0};
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int x = it.a + (q & (kTile - 1)), y = it.b + q / kTile;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const double f1 = P.f[RECON_F_F1][d], f2 = P.f[RECON_F_F2][d];
            const double m1 = c.b00 * f1 + c.b10 * f2;
            const double m2 = c.b01 * f1 + c.b11 * f2;
            const double rho_cf = (m1 * c.r - m2) / c.c_rho;
            const double a = (m1 * c.P2 - m2 * c.P1) / c.a_w;
            const double b = (m2 * c.psi1 - m1 * c.psi2) / c.a_w;
            const T rr = T(rho_cf) + P.f[RECON_F_DIV_RHO][d];
            const T a2 = T(a * a);
            const T rz = T(a * b) + P.f[RECON_F_DIV_Z][d];
            P.f[RECON_F_RHS_RHO][d] = rr;
            P.f[RECON_F_A2][d] = a2;
            P.f[RECON_F_RHS_Z][d] = rz;
            acc[0] += (double)a2;
            acc[1] += (double)rz * (double)rz;
        }
        block_sum<2>(acc, red);
        double tot[2];
        if (item_reduce<2>(L, w, it.slice, acc, tot)) {
            SliceState& so = S[it.slice];
            so.abar2 = tot[0] / ((double)g.nx * (double)g.ny);
            so.bb = tot[1];
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// PCG for [diag(a^2) + beta~ L] z = rhs
// --------------------------------------------------------------------------

// stencil tile of a vector with its 4-neighbour halo (periodic)
template <typename T, typename F>
__device__ __forceinline__ void load_halo(T (*sm)[kTile + 2], const SliceGeom& g, const Item& it, F value) {
    for (int q = threadIdx.x; q < (kTile + 2) * (kTile + 2); q += blockDim.x) {
        const int ly = q / (kTile + 2), lx = q - ly * (kTile + 2);
        const bool corner = (ly == 0 || ly == kTile + 1) && (lx == 0 || lx == kTile + 1);
        if (corner) continue;
        const int gy = wrap(it.b - 1 + ly, g.ny), gx = wrap(it.a - 1 + lx, g.nx);
        sm[ly][lx] = value(g.off + (long long)gy * g.pitch + gx);
    }
}

template <typename T>
__device__ __forceinline__ T lap5(const T (*sm)[kTile + 2], int ly, int lx) {
    const T c = sm[ly + 1][lx + 1];
    return (T(4) * c - sm[ly + 1][lx] - sm[ly + 1][lx + 2]) - (sm[ly][lx + 1] + sm[ly + 2][lx + 1]);
}

__device__ __forceinline__ bool cg_skip(const SliceState& st) { return !st.active || st.cg_done; }

template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_cg_init(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                             SliceState* S, Ptrs<T> P, int* pending) {
    __shared__ T sm[kTile + 2][kTile + 2];
    __shared__ double red[32];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState st = S[it.slice];
        if (!st.active) continue;
        const SliceGeom g = G[it.slice];
        account(P.acct, KF_CG_INIT, tile_px(g, it) * 4 * (long long)sizeof(T));
        const T* z = P.f[RECON_F_Z];
        load_halo<T>(sm, g, it, [&](long long d) { return z[d]; });
        __syncthreads();
        const T bt = T(st.beta_t);
        double acc[1] = {0.0};
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int lx = q & (kTile - 1), ly = q / kTile;
            const int x = it.a + lx, y = it.b + ly;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const T Mz = P.f[RECON_F_A2][d] * sm[ly + 1][lx + 1] + bt * lap5<T>(sm, ly, lx);
            const T r = P.f[RECON_F_RHS_Z][d] - Mz;
            P.f[RECON_F_CG_R][d] = r;
            acc[0] += (double)r * (double)r;
        }
        block_sum<1>(acc, red);
        double tot[1];
        if (item_reduce<1>(L, w, it.slice, acc, tot)) {
            SliceState& so = S[it.slice];
            const double tol2 = C[it.slice].cg_tol * C[it.slice].cg_tol;
            so.rr = tot[0];
            so.rr0 = tot[0];
            so.cg_it = 0;
            so.ry = 0.0;
            so.betacg = 0.0;
            so.cg_done = (so.bb == 0.0 || !(tot[0] > tol2 * so.bb)) ? 1 : 0;
            if (!so.cg_done) atomicAdd(pending, 1);
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_cg_matvec(ItemList L, const SliceGeom* G, SliceState* S,
                                                               Ptrs<T> P, int par) {
    __shared__ T sm[kTile + 2][kTile + 2];
    __shared__ double red[32];
    const T* pold = P.f[par ? RECON_F_CG_P1 : RECON_F_CG_P0];
    T* pnew = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    const T* yv = P.f[RECON_F_CG_Y];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState st = S[it.slice];
        if (cg_skip(st)) continue;
        const SliceGeom g = G[it.slice];
        account(P.acct, KF_CG_MATVEC, tile_px(g, it) * 5 * (long long)sizeof(T));
        const bool first = st.cg_it == 0;
        const T bc = T(st.betacg);
        load_halo<T>(sm, g, it, [&](long long d) { return first ? yv[d] : yv[d] + bc * pold[d]; });
        __syncthreads();
        const T bt = T(st.beta_t);
        double acc[1] = {0.0};
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int lx = q & (kTile - 1), ly = q / kTile;
            const int x = it.a + lx, y = it.b + ly;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const T p = sm[ly + 1][lx + 1];
            const T qv = P.f[RECON_F_A2][d] * p + bt * lap5<T>(sm, ly, lx);
            pnew[d] = p;
            P.f[RECON_F_CG_Q][d] = qv;
            acc[0] += (double)p * (double)qv;
        }
        block_sum<1>(acc, red);
        double tot[1];
        if (item_reduce<1>(L, w, it.slice, acc, tot)) {
            SliceState& so = S[it.slice];
            so.pq = tot[0];
            so.alpha = tot[0] > 0.0 ? so.ry / tot[0] : 0.0;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_cg_update(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                               SliceState* S, Ptrs<T> P, int par, int* pending) {
    __shared__ double red[32];
    const T* p = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState st = S[it.slice];
        if (cg_skip(st)) continue;
        const SliceGeom g = G[it.slice];
        account(P.acct, KF_CG_UPDATE, tile_px(g, it) * 6 * (long long)sizeof(T));
        const T al = T(st.alpha);
        double acc[1] = {0.0};
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int x = it.a + (q & (kTile - 1)), y = it.b + q / kTile;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            P.f[RECON_F_Z][d] += al * p[d];
            const T r = P.f[RECON_F_CG_R][d] - al * P.f[RECON_F_CG_Q][d];
            P.f[RECON_F_CG_R][d] = r;
            acc[0] += (double)r * (double)r;
        }
        block_sum<1>(acc, red);
        double tot[1];
        if (item_reduce<1>(L, w, it.slice, acc, tot)) {
            SliceState& so = S[it.slice];
            const SliceConst& c = C[it.slice];
            so.rr = tot[0];
            so.cg_it += 1;
            const bool conv = !(tot[0] > c.cg_tol * c.cg_tol * so.bb);
            if (conv || so.cg_it >= c.cg_max) {
                so.cg_done = 1;
                atomicSub(pending, 1);
            }
        }
        __syncthreads();
    }
}

__global__ void k_next_beta(int n, const SliceConst* C, SliceState* S) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SliceState& st = S[s];
    if (!st.active) return;
    const SliceConst& c = C[s];
    st.k += 1;
    st.beta *= c.kappa;
    st.beta_t = c.tau * st.beta;
    st.thr_d = c.lambda / st.beta;
    st.thr_f = (float)st.thr_d;
    st.active = st.k < c.iters;
}

__global__ void k_reset_state(int n, const SliceConst* C, SliceState* S) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const SliceConst& c = C[s];
    SliceState st = {};
    st.beta = c.beta0;
    st.beta_t = c.tau * c.beta0;
    st.thr_d = c.lambda / c.beta0;
    st.thr_f = (float)st.thr_d;
    st.k = 0;
    st.active = c.iters > 0;
    st.cg_done = 1;
    S[s] = st;
}

// --------------------------------------------------------------------------
// Z = Z_w (Z^m / Z_w^m)^(1/m) by FP64 Newton on y^m = z (Sec. II-D: Z is the
// m-th root of Z^m); Z = 1 where z <= 0.
// --------------------------------------------------------------------------

__device__ __forceinline__ double mth_root_newton(double z, double m) {
    double y = (double)powf((float)z, (float)(1.0 / m));  // FP32 start
    for (int i = 0; i < 3; ++i) {
        const double ym = pow(y, m);
        y = y - (ym - z) / (m * ym / y);
    }
    return y;
}

template <typename T>
__global__ void k_extract(ItemList L, const SliceGeom* G, Ptrs<T> P, float* Z, float* rhoe, float* f1, float* f2,
                          double zw, double m) {
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceGeom g = G[it.slice];
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int x = it.a + (q & (kTile - 1)), y = it.b + q / kTile;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const long long e = g.ext_off + (long long)y * g.nx + x;
            if (Z) {
                const double z = P.f[RECON_F_Z][d];
                Z[e] = z > 0.0 ? (float)(zw * mth_root_newton(z, m)) : 1.0f;
            }
            if (rhoe) rhoe[e] = (float)P.f[RECON_F_RHO][d];
            if (f1) f1[e] = (float)P.f[RECON_F_F1][d];
            if (f2) f2[e] = (float)P.f[RECON_F_F2][d];
        }
    }
}

// ==========================================================================
// host side
// ==========================================================================

namespace {

template <typename T>
Ptrs<T> ptrs(Ctx& c) {
    Ptrs<T> p;
    for (int i = 0; i < kNumFields; ++i) p.f[i] = static_cast<T*>(c.field[i]);
    for (int i = 0; i < kNumSpectra; ++i) p.s[i] = static_cast<cplx<T>*>(c.spec[i]);
    p.acct = c.d_acct;
    return p;
}

int grid_for(const Ctx& c, int work) {
    const int cap = c.sm_count * 8;
    return work < cap ? (work > 0 ? work : 1) : cap;
}

template <typename T>
int fft_smem_bytes(const Ctx& c) {
    const int buf = kRowBudget + 64;
    const int tw = c.max_nx > c.max_ny ? c.max_nx : c.max_ny;
    return (2 * buf + tw) * (int)sizeof(cplx<T>);
}

template <typename T>
int fft_solve(Ctx& c, const FftJobs& J, int mode) {
    const Ptrs<T> P = ptrs<T>(c);
    const int smem = fft_smem_bytes<T>(c);
    const int buf = kRowBudget + 64;
    if (mode == 0) {
        FamTimer t(c, KF_ROWS_FWD);
        k_rows_fwd<T, 0><<<grid_for(c, c.rows.n * J.n), kFftThreads, smem, c.stream>>>(c.rows.view(), c.d_geom,
                                                                                       c.d_state, P, J, buf);
    } else {
        FamTimer t(c, KF_ROWS_FWD_PRE);
        k_rows_fwd<T, 1><<<grid_for(c, c.rows.n * J.n), kFftThreads, smem, c.stream>>>(c.rows.view(), c.d_geom,
                                                                                       c.d_state, P, J, buf);
    }
    {
        FamTimer t(c, mode ? KF_COLS_PRE : KF_COLS);
        k_cols<T><<<grid_for(c, c.cols.n * J.n), kFftThreads, smem, c.stream>>>(c.cols.view(), c.d_geom, c.d_const,
                                                                               c.d_state, P, J, buf);
    }
    if (mode == 0) {
        FamTimer t(c, KF_ROWS_INV);
        k_rows_inv<T, 0><<<grid_for(c, c.rows.n * J.n), kFftThreads, smem, c.stream>>>(c.rows.view(), c.d_geom,
                                                                                       c.d_state, P, J, buf);
    } else {
        FamTimer t(c, KF_ROWS_INV_PRE);
        k_rows_inv<T, 1><<<grid_for(c, c.rows.n * J.n), kFftThreads, smem, c.stream>>>(c.rows.view(), c.d_geom,
                                                                                       c.d_state, P, J, buf);
    }
    c.launches += 3;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int set_fft_smem(Ctx& c) {
    const int smem = fft_smem_bytes<T>(c);
    RECON_CUDA(cudaFuncSetAttribute(k_rows_fwd<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_rows_fwd<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_rows_inv<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_rows_inv<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return RECON_OK;
}

FftJobs jobs1(int in, int spec, int out, int coef) {
    FftJobs J{};
    J.n = 1;
    J.in[0] = in;
    J.spec[0] = spec;
    J.out[0] = out;
    J.coef[0] = coef;
    return J;
}

template <typename T>
int op_thr_rhs(Ctx& c, bool stats) {
    const Ptrs<T> P = ptrs<T>(c);
    FamTimer t(c, KF_THR_RHS);
    if (stats)
        k_thr_rhs<T, true><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom,
                                                                                     c.d_const, c.d_state, P);
    else
        k_thr_rhs<T, false><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom,
                                                                                      c.d_const, c.d_state, P);
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int op_solve_f(Ctx& c) {
    int rc;
    if (c.prm[0].order == 0) {
        FftJobs J{};
        J.n = 2;
        J.in[0] = RECON_F_RHS_F1; J.spec[0] = 0; J.out[0] = RECON_F_F1; J.coef[0] = 0;
        J.in[1] = RECON_F_RHS_F2; J.spec[1] = 1; J.out[1] = RECON_F_F2; J.coef[1] = 1;
        return fft_solve<T>(c, J, 0);
    }
    if ((rc = fft_solve<T>(c, jobs1(RECON_F_RHS_F1, 0, RECON_F_F1, 0), 0))) return rc;
    k_gs_fix<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, c.d_const,
                                                                         c.d_state, ptrs<T>(c));
    c.launches += 1;
    return fft_solve<T>(c, jobs1(RECON_F_RHS_F2, 1, RECON_F_F2, 1), 0);
}

template <typename T>
int op_synth(Ctx& c) {
    FamTimer t(c, KF_SYNTH);
    k_synth<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, c.d_const,
                                                                        c.d_state, ptrs<T>(c));
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int op_solve_z(Ctx& c) {
    const Ptrs<T> P = ptrs<T>(c);
    RECON_CUDA(cudaMemsetAsync(c.d_cg_pending, 0, sizeof(int), c.stream));
    FamTimer t0(c, KF_CG_INIT);
    k_cg_init<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, c.d_const,
                                                                          c.d_state, P, c.d_cg_pending);
    c.launches += 1;
    const FftJobs pre = jobs1(RECON_F_CG_R, 0, RECON_F_CG_Y, 3);
    int rc = fft_solve<T>(c, pre, 1);
    if (rc) return rc;
    int cap = 0;
    for (const auto& p : c.prm) cap = p.cg_max_iters > cap ? p.cg_max_iters : cap;
    int par = c.cg_parity;
    for (int it = 0; it < cap; ++it) {
        {
            FamTimer t(c, KF_CG_MATVEC);
            k_cg_matvec<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom,
                                                                                    c.d_state, P, par);
        }
        {
            FamTimer t(c, KF_CG_UPDATE);
            k_cg_update<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(
                c.tiles.view(), c.d_geom, c.d_const, c.d_state, P, par, c.d_cg_pending);
        }
        c.launches += 2;
        if ((rc = fft_solve<T>(c, pre, 1))) return rc;
        par ^= 1;
        if ((it & 3) == 3 || it == cap - 1) {
            RECON_CUDA(cudaMemcpyAsync(c.h_cg_pending, c.d_cg_pending, sizeof(int), cudaMemcpyDeviceToHost,
                                       c.stream));
            RECON_CUDA(cudaStreamSynchronize(c.stream));
            if (*c.h_cg_pending <= 0) break;
        }
    }
    c.cg_parity = par;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int op_next_beta(Ctx& c) {
    k_next_beta<<<(c.n + 127) / 128, 128, 0, c.stream>>>(c.n, c.d_const, c.d_state);
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int iterate_t(Ctx& c, bool stats) {
    int rc;
    if ((rc = op_thr_rhs<T>(c, stats))) return rc;
    if ((rc = op_solve_f<T>(c))) return rc;
    if ((rc = op_synth<T>(c))) return rc;
    if ((rc = fft_solve<T>(c, jobs1(RECON_F_RHS_RHO, 2, RECON_F_RHO, 2), 0))) return rc;
    if ((rc = op_solve_z<T>(c))) return rc;
    return op_next_beta<T>(c);
}

template <typename T>
int init_maps_t(Ctx& c) {
    k_reset_state<<<(c.n + 127) / 128, 128, 0, c.stream>>>(c.n, c.d_const, c.d_state);
    k_init<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, c.d_const,
                                                                        ptrs<T>(c));
    c.launches += 2;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int load_t(Ctx& c, const float* lo, const float* hi) {
    k_load<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(
        c.tiles.view(), c.d_geom, c.d_const, lo, hi, static_cast<T*>(c.field[RECON_F_MUL]),
        static_cast<T*>(c.field[RECON_F_MUH]));
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int extract_t(Ctx& c, float* Z, float* rhoe, float* f1, float* f2) {
    k_extract<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, ptrs<T>(c), Z,
                                                                           rhoe, f1, f2, water_z(), z_exponent());
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int op_t(Ctx& c, int op) {
    switch (op) {
        case RECON_OP_INIT: return init_maps_t<T>(c);
        case RECON_OP_THRESH_RHS: return op_thr_rhs<T>(c, false);
        case RECON_OP_SOLVE_F: return op_solve_f<T>(c);
        case RECON_OP_SYNTH: return op_synth<T>(c);
        case RECON_OP_SOLVE_RHO: return fft_solve<T>(c, jobs1(RECON_F_RHS_RHO, 2, RECON_F_RHO, 2), 0);
        case RECON_OP_SOLVE_Z: return op_solve_z<T>(c);
        case RECON_OP_NEXT_BETA: return op_next_beta<T>(c);
        default: set_error("unknown operator"); return RECON_EINVAL;
    }
}

int alloc_dev(Ctx& c, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        return RECON_ENOMEM;
    }
    c.allocations.push_back(*p);
    return RECON_OK;
}

int upload_list(Ctx& c, DevItemList& L) {
    int rc;
    L.n = (int)L.h_items.size();
    if ((rc = alloc_dev(c, (void**)&L.items, sizeof(Item) * L.h_items.size()))) return rc;
    if ((rc = alloc_dev(c, (void**)&L.lo, sizeof(int) * c.n))) return rc;
    if ((rc = alloc_dev(c, (void**)&L.cnt, sizeof(int) * c.n))) return rc;
    if ((rc = alloc_dev(c, (void**)&L.partials, sizeof(double) * kMaxPartials * L.h_items.size()))) return rc;
    if ((rc = alloc_dev(c, (void**)&L.counters, sizeof(unsigned) * c.n))) return rc;
    RECON_CUDA(cudaMemcpy(L.items, L.h_items.data(), sizeof(Item) * L.h_items.size(), cudaMemcpyHostToDevice));
    RECON_CUDA(cudaMemcpy(L.lo, L.h_lo.data(), sizeof(int) * c.n, cudaMemcpyHostToDevice));
    RECON_CUDA(cudaMemcpy(L.cnt, L.h_cnt.data(), sizeof(int) * c.n, cudaMemcpyHostToDevice));
    RECON_CUDA(cudaMemset(L.counters, 0, sizeof(unsigned) * c.n));
    return RECON_OK;
}

}  // namespace

int solver_setup(Ctx& c) {
    int rc;
    int dev = 0;
    RECON_CUDA(cudaGetDevice(&dev));
    RECON_CUDA(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev));
    c.elem = c.precision == 1 ? sizeof(float) : sizeof(double);
    // placement
    c.sg.resize(c.n);
    long long off = 0, coff = 0, ext = 0;
    c.max_nx = c.max_ny = 0;
    for (int s = 0; s < c.n; ++s) {
        SliceGeom& g = c.sg[s];
        g.nx = c.geo[s].nx;
        g.ny = c.geo[s].ny;
        g.pitch = (g.nx + 31) / 32 * 32;
        g.nh = g.nx / 2 + 1;
        g.cpitch = (g.nh + 15) / 16 * 16;
        g.off = off;
        g.coff = coff;
        g.ext_off = ext;
        off += (long long)g.ny * g.pitch;
        coff += (long long)g.ny * g.cpitch;
        ext += (long long)g.ny * g.nx;
        c.max_nx = g.nx > c.max_nx ? g.nx : c.max_nx;
        c.max_ny = g.ny > c.max_ny ? g.ny : c.max_ny;
    }
    c.pool_elems = off;
    c.spec_elems = coff;
    c.ext_elems = ext;
    // item lists
    c.tiles.h_lo.assign(c.n, 0); c.tiles.h_cnt.assign(c.n, 0);
    c.rows.h_lo.assign(c.n, 0); c.rows.h_cnt.assign(c.n, 0);
    c.cols.h_lo.assign(c.n, 0); c.cols.h_cnt.assign(c.n, 0);
    for (int s = 0; s < c.n; ++s) {
        const SliceGeom& g = c.sg[s];
        c.tiles.h_lo[s] = (int)c.tiles.h_items.size();
        for (int ty = 0; ty < g.ny; ty += kTile)
            for (int tx = 0; tx < g.nx; tx += kTile) c.tiles.h_items.push_back(Item{s, tx, ty, 0});
        c.tiles.h_cnt[s] = (int)c.tiles.h_items.size() - c.tiles.h_lo[s];
        c.rows.h_lo[s] = (int)c.rows.h_items.size();
        const int npairs = (g.ny + 1) / 2;
        int per = kRowBudget / g.nx;
        if (per < 1) per = 1;
        for (int p0 = 0; p0 < npairs; p0 += per)
            c.rows.h_items.push_back(Item{s, p0, (npairs - p0 < per ? npairs - p0 : per), 0});
        c.rows.h_cnt[s] = (int)c.rows.h_items.size() - c.rows.h_lo[s];
        c.cols.h_lo[s] = (int)c.cols.h_items.size();
        int pc = kRowBudget / g.ny;
        if (pc > 16) pc = 16;
        if (pc < 1) pc = 1;
        for (int c0 = 0; c0 < g.nh; c0 += pc) c.cols.h_items.push_back(Item{s, c0, (g.nh - c0 < pc ? g.nh - c0 : pc), 0});
        c.cols.h_cnt[s] = (int)c.cols.h_items.size() - c.cols.h_lo[s];
    }
    if ((rc = upload_list(c, c.tiles)) || (rc = upload_list(c, c.rows)) || (rc = upload_list(c, c.cols))) return rc;
    // constants
    std::vector<SliceConst> hc(c.n);
    c.tab.resize(c.n);
    for (int s = 0; s < c.n; ++s) {
        const recon_params& p = c.prm[s];
        const Tables t = make_tables(p);
        c.tab[s] = t;
        SliceConst& k = hc[s];
        k.a00 = t.a[0][0]; k.a01 = t.a[0][1]; k.a10 = t.a[1][0]; k.a11 = t.a[1][1];
        k.b00 = t.b[0][0]; k.b01 = t.b[0][1]; k.b10 = t.b[1][0]; k.b11 = t.b[1][1];
        k.P1 = t.P[0]; k.P2 = t.P[1]; k.psi1 = t.psi[0]; k.psi2 = t.psi[1];
        k.r = t.r; k.c_f1 = t.c_f[0]; k.c_f2 = t.c_f[1]; k.c12 = t.c12; k.c_rho = t.c_rho; k.a_w = t.a_w;
        k.det = t.det; k.inv_S = 1.0 / t.S; k.zclip_hi = t.zclip_hi; k.rho_air = p.rho_air;
        k.lambda = p.lambda; k.beta0 = p.beta0; k.tau = p.tau;
        k.kappa = p.kappa > 0 ? p.kappa : (p.iters > 0 ? std::pow(p.beta_max / p.beta0, 1.0 / p.iters) : 1.0);
        k.cg_tol = p.cg_tol; k.iters = p.iters; k.order = p.order; k.cg_max = p.cg_max_iters;
    }
    if ((rc = alloc_dev(c, (void**)&c.d_geom, sizeof(SliceGeom) * c.n))) return rc;
    if ((rc = alloc_dev(c, (void**)&c.d_const, sizeof(SliceConst) * c.n))) return rc;
    if ((rc = alloc_dev(c, (void**)&c.d_state, sizeof(SliceState) * c.n))) return rc;
    RECON_CUDA(cudaMemcpy(c.d_geom, c.sg.data(), sizeof(SliceGeom) * c.n, cudaMemcpyHostToDevice));
    RECON_CUDA(cudaMemcpy(c.d_const, hc.data(), sizeof(SliceConst) * c.n, cudaMemcpyHostToDevice));
    RECON_CUDA(cudaMemset(c.d_state, 0, sizeof(SliceState) * c.n));
    // pools
    for (int f = 0; f < kNumFields; ++f) {
        if ((rc = alloc_dev(c, &c.field[f], c.elem * c.pool_elems))) return rc;
        RECON_CUDA(cudaMemset(c.field[f], 0, c.elem * c.pool_elems));
    }
    for (int f = 0; f < kNumSpectra; ++f)
        if ((rc = alloc_dev(c, &c.spec[f], 2 * c.elem * c.spec_elems))) return rc;
    for (int i = 0; i < 2; ++i)
        if ((rc = alloc_dev(c, (void**)&c.d_stage[i], sizeof(float) * c.ext_elems))) return rc;
    if ((rc = alloc_dev(c, (void**)&c.d_cg_pending, sizeof(int)))) return rc;
    if ((rc = alloc_dev(c, (void**)&c.d_acct, sizeof(unsigned long long) * KF_COUNT))) return rc;
    RECON_CUDA(cudaMemset(c.d_acct, 0, sizeof(unsigned long long) * KF_COUNT));
    RECON_CUDA(cudaMallocHost((void**)&c.h_cg_pending, sizeof(int)));
    if (c.precision == 1) return set_fft_smem<float>(c);
    return set_fft_smem<double>(c);
}

int solver_load_images(Ctx& c, const float* lo, const float* hi, int /*on_device*/) {
    return c.precision == 1 ? load_t<float>(c, lo, hi) : load_t<double>(c, lo, hi);
}

int solver_init_maps(Ctx& c) { return c.precision == 1 ? init_maps_t<float>(c) : init_maps_t<double>(c); }

int solver_iterate(Ctx& c, bool stats) {
    return c.precision == 1 ? iterate_t<float>(c, stats) : iterate_t<double>(c, stats);
}

int solver_op(Ctx& c, int op) { return c.precision == 1 ? op_t<float>(c, op) : op_t<double>(c, op); }

int solver_extract(Ctx& c, float* Z, float* rhoe, float* f1, float* f2, int /*on_device*/) {
    return c.precision == 1 ? extract_t<float>(c, Z, rhoe, f1, f2) : extract_t<double>(c, Z, rhoe, f1, f2);
}

FamTimer::FamTimer(Ctx& ctx, int f) : c(ctx), fam(f) {
    c.fam_launches[f] += 1;
    if (!(c.prof_mask & (1u << f))) return;
    for (cudaEvent_t* ev : {&b, &e}) {
        if (!c.ev_pool.empty()) {
            *ev = c.ev_pool.back();
            c.ev_pool.pop_back();
        } else if (cudaEventCreate(ev) != cudaSuccess) {
            *ev = nullptr;
        }
    }
    if (b && e) cudaEventRecord(b, c.stream);
}

FamTimer::~FamTimer() {
    if (b && e) {
        cudaEventRecord(e, c.stream);
        c.ev_used.push_back({fam, {b, e}});
    } else {
        if (b) c.ev_pool.push_back(b);
        if (e) c.ev_pool.push_back(e);
    }
}

int solver_profile_read(Ctx& c, double* ms, long long* launches, unsigned long long* bytes) {
    RECON_CUDA(cudaStreamSynchronize(c.stream));
    for (int f = 0; f < KF_COUNT; ++f) {
        if (ms) ms[f] = 0.0;
        if (launches) launches[f] = c.fam_launches[f];
        c.fam_launches[f] = 0;
    }
    for (auto& u : c.ev_used) {
        float t = 0.f;
        RECON_CUDA(cudaEventElapsedTime(&t, u.second.first, u.second.second));
        if (ms) ms[u.first] += t;
        c.ev_pool.push_back(u.second.first);
        c.ev_pool.push_back(u.second.second);
    }
    c.ev_used.clear();
    std::vector<unsigned long long> h(KF_COUNT);
    RECON_CUDA(cudaMemcpy(h.data(), c.d_acct, sizeof(unsigned long long) * KF_COUNT, cudaMemcpyDeviceToHost));
    RECON_CUDA(cudaMemset(c.d_acct, 0, sizeof(unsigned long long) * KF_COUNT));
    if (bytes)
        for (int f = 0; f < KF_COUNT; ++f) bytes[f] = h[f];
    return RECON_OK;
}

int solver_read_state(Ctx& c, std::vector<SliceState>& out) {
    out.resize(c.n);
    RECON_CUDA(cudaMemcpyAsync(out.data(), c.d_state, sizeof(SliceState) * c.n, cudaMemcpyDeviceToHost, c.stream));
    RECON_CUDA(cudaStreamSynchronize(c.stream));
    return RECON_OK;
}

}  // namespace recon
