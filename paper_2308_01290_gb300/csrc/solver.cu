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
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <memory>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "fft.cuh"

namespace recon {

template <typename T>
struct Ptrs {
    T* f[kNumFields];
    cplx<T>* s[kNumSpectra];
    unsigned long long* acct;   // algorithmic bytes per kernel family
    const T* sym;               // symbol tables 4 sin^2(pi t / N)
};

// Adds the algorithmic bytes of one processed item to its family's counter.
__device__ __forceinline__ void account(unsigned long long* acct, int fam, long long bytes) {
    if (threadIdx.x == 0) atomicAdd(acct + fam, (unsigned long long)bytes);
}

template <typename T>
struct TileH;
template <>
struct TileH<float> {
    static constexpr int v = kTileHFloat;
};
template <>
struct TileH<double> {
    static constexpr int v = kTileHDouble;
};

template <typename T>
__device__ __forceinline__ long long tile_px(const SliceGeom& g, const Item& it) {
    constexpr int TH = TileH<T>::v;
    const int w = g.nx - it.a < kTileW ? g.nx - it.a : kTileW;
    const int h = g.ny - it.b < TH ? g.ny - it.b : TH;
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

// a*b - c*d with the product c*d split exactly (FMA two-product), so the
// difference of two nearly equal products keeps its precision.
template <typename T>
__device__ __forceinline__ T diff_of_products(T a, T b, T c, T d) {
    const T cd = c * d;
    const T err = fma(c, d, -cd);
    return fma(a, b, -cd) - err;
}

// Jacobi scaling of the Z^m preconditioner: sqrt(num / (a2 + b4)), with
// sqrt(num) passed in.
__device__ __forceinline__ float dscale(float sqrt_num, float a2, float b4) { return sqrt_num * rsqrtf(a2 + b4); }
__device__ __forceinline__ double dscale(double sqrt_num, double a2, double b4) { return sqrt_num / sqrt(a2 + b4); }

// 1 / (nx ny) in the kernel's precision.
template <typename T>
__device__ __forceinline__ T inv_n_of(const SliceGeom& g) {
    if constexpr (sizeof(T) == 4)
        return g.inv_n;
    else
        return 1.0 / ((double)g.nx * (double)g.ny);
}

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
        for (int q = threadIdx.x; q < kTileW * TileH<T>::v; q += blockDim.x) {
            const int x = it.a + (q & (kTileW - 1)), y = it.b + q / kTileW;
            if (x >= g.nx || y >= g.ny) continue;
            const long long e = g.ext_off + (long long)y * g.nx + x;
            const long long d = g.off + (long long)y * g.pitch + x;
            muL[d] = T((double)lo[e] * s);
            muH[d] = T((double)hi[e] * s);
        }
    }
}

// The per-pixel initialisation of Algorithm 1 from the normalised image pair
// (uL, uH), in FP64: f by Cramer's rule on eq. lac_EL / lac_EH, the synthesis
// eq. mac_E1 / mac_E2, and the closed forms eq. rho_e and eq. Z_m
// (normalised, reading R3; z set to water where a = 0 or rho_e < rho_air and
// clipped to the Z range, reading R16).  This is also the two-step
// image-based comparator of Sec. III.
__device__ __forceinline__ void init_pixel(const SliceConst& c, double uL, double uH, double& f1, double& f2,
                                           double& rho, double& z) {
    f1 = (c.a11 * uL - c.a10 * uH) / c.det;
    f2 = (c.a00 * uH - c.a01 * uL) / c.det;
    const double m1 = c.b00 * f1 + c.b10 * f2;
    const double m2 = c.b01 * f1 + c.b11 * f2;
    rho = (m1 * c.r - m2) / c.c_rho;
    const double a = (m1 * c.P2 - m2 * c.P1) / c.a_w;
    const double b = (m2 * c.psi1 - m1 * c.psi2) / c.a_w;
    z = 1.0;
    if (a != 0.0 && rho >= c.rho_air) z = fmin(fmax(b / a, 0.0), c.zclip_hi);
}

template <typename T>
__global__ void k_init(ItemList L, const SliceGeom* G, const SliceConst* C, Ptrs<T> P) {
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceGeom g = G[it.slice];
        const SliceConst c = C[it.slice];
        for (int q = threadIdx.x; q < kTileW * TileH<T>::v; q += blockDim.x) {
            const int x = it.a + (q & (kTileW - 1)), y = it.b + q / kTileW;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            double f1, f2, rho, z;
            init_pixel(c, P.f[RECON_F_MUL][d], P.f[RECON_F_MUH][d], f1, f2, rho, z);
            P.f[RECON_F_F1][d] = T(f1);
            P.f[RECON_F_F2][d] = T(f2);
            P.f[RECON_F_RHO][d] = T(rho);
            P.f[RECON_F_Z][d] = T(z);
        }
    }
}

// --------------------------------------------------------------------------
// tiles in shared memory: kTileW x TH pixels plus a one-pixel halo; the
// interior starts at a 16-byte boundary (column OFF) so rows move as 16-byte
// vectors; left halo at column OFF - 1, right halo at OFF + kTileW.
// --------------------------------------------------------------------------

template <typename T>
struct TileDim {
    static constexpr int VN = 16 / (int)sizeof(T);   // elements per 16-byte vector
    static constexpr int OFF = VN;
    static constexpr int TH = TileH<T>::v;
    static constexpr int SW = OFF + kTileW + VN;     // row stride
};

template <typename T>
struct alignas(16) Pack {
    T v[TileDim<T>::VN];
};

template <typename T, int NM>
struct Vals {
    T v[NM];
};
template <typename T, int NM>
struct PVals {
    Pack<T> p[NM];
};


// Load NM maps of one tile with halo.  vect(d) gives the NM 16-byte packs at
// element offset d (16-byte aligned), scal(d) the NM scalars at d.
template <typename T, int NM, typename FS, typename FV>
__device__ __forceinline__ void load_tile(T (*sm)[TileDim<T>::TH + 2][TileDim<T>::SW], const SliceGeom& g, int tx0,
                                          int ty0, FS scal, FV vect) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, TH = TileDim<T>::TH;
    if (NM > 2 && tx0 + kTileW <= g.nx) {
        // many maps: round by round (registers)
        constexpr int VR = kTileW / VN;
        for (int q = threadIdx.x; q < (TH + 2) * VR; q += blockDim.x) {
            const int ly = q / VR, lx = (q - ly * VR) * VN;
            const int gy = wrap(ty0 - 1 + ly, g.ny);
            const PVals<T, NM> pv = vect(g.off + (long long)gy * g.pitch + tx0 + lx);
#pragma unroll
            for (int m = 0; m < NM; ++m) *reinterpret_cast<Pack<T>*>(&sm[m][ly][OFF + lx]) = pv.p[m];
        }
        for (int q = threadIdx.x; q < 2 * (TH + 2); q += blockDim.x) {
            const int ly = q >> 1, side = q & 1;
            const int gy = wrap(ty0 - 1 + ly, g.ny);
            const int gx = side ? wrap(tx0 + kTileW, g.nx) : wrap(tx0 - 1, g.nx);
            const Vals<T, NM> sv = scal(g.off + (long long)gy * g.pitch + gx);
#pragma unroll
            for (int m = 0; m < NM; ++m) sm[m][ly][side ? OFF + kTileW : OFF - 1] = sv.v[m];
        }
    } else if (tx0 + kTileW <= g.nx) {
        // every load of the tile (vector rounds and halo) is issued before
        // the first store to shared memory; blockDim.x == kStencilThreads
        constexpr int VR = kTileW / VN, NV = (TH + 2) * VR;
        constexpr int RV = (NV + kStencilThreads - 1) / kStencilThreads;
        PVals<T, NM> pv[RV];
#pragma unroll
        for (int u = 0; u < RV; ++u) {
            const int q = threadIdx.x + u * kStencilThreads;
            if (q < NV) {
                const int ly = q / VR, lx = (q - ly * VR) * VN;
                const int gy = wrap(ty0 - 1 + ly, g.ny);
                pv[u] = vect(g.off + (long long)gy * g.pitch + tx0 + lx);
            }
        }
        const int hq = threadIdx.x;
        const bool halo = hq < 2 * (TH + 2);
        Vals<T, NM> sv;
        if (halo) {
            const int ly = hq >> 1, side = hq & 1;
            const int gy = wrap(ty0 - 1 + ly, g.ny);
            const int gx = side ? wrap(tx0 + kTileW, g.nx) : wrap(tx0 - 1, g.nx);
            sv = scal(g.off + (long long)gy * g.pitch + gx);
        }
#pragma unroll
        for (int u = 0; u < RV; ++u) {
            const int q = threadIdx.x + u * kStencilThreads;
            if (q < NV) {
                const int ly = q / VR, lx = (q - ly * VR) * VN;
#pragma unroll
                for (int m = 0; m < NM; ++m) *reinterpret_cast<Pack<T>*>(&sm[m][ly][OFF + lx]) = pv[u].p[m];
            }
        }
        if (halo) {
            const int ly = hq >> 1, side = hq & 1;
#pragma unroll
            for (int m = 0; m < NM; ++m) sm[m][ly][side ? OFF + kTileW : OFF - 1] = sv.v[m];
        }
    } else {
        for (int q = threadIdx.x; q < (TH + 2) * (kTileW + 2); q += blockDim.x) {
            const int ly = q / (kTileW + 2), lx = q - ly * (kTileW + 2);
            const int gy = wrap(ty0 - 1 + ly, g.ny), gx = wrap(tx0 - 1 + lx, g.nx);
            const Vals<T, NM> sv = scal(g.off + (long long)gy * g.pitch + gx);
#pragma unroll
            for (int m = 0; m < NM; ++m) sm[m][ly][OFF - 1 + lx] = sv.v[m];
        }
    }
}

template <typename T>
__device__ __forceinline__ Pack<T> ldv(const T* p, long long d) {
    return *reinterpret_cast<const Pack<T>*>(p + d);
}
template <typename T>
__device__ __forceinline__ void stv(T* p, long long d, const Pack<T>& v) {
    *reinterpret_cast<Pack<T>*>(p + d) = v;
}

// Visit the pixels of a tile VN at a time: fn(d0, e_count, full) with d0 the
// element offset of the first pixel of the vector; `full` when all VN lie
// inside the image.
template <typename T, typename F>
__device__ __forceinline__ void for_tile_vectors(const SliceGeom& g, const Item& it, F fn) {
    constexpr int VN = TileDim<T>::VN, VR = kTileW / VN;
    for (int q = threadIdx.x; q < TileDim<T>::TH * VR; q += blockDim.x) {
        const int ly = q / VR, lx0 = (q - ly * VR) * VN;
        const int y = it.b + ly, x0 = it.a + lx0;
        if (y >= g.ny || x0 >= g.nx) continue;
        const int cnt = g.nx - x0 < VN ? g.nx - x0 : VN;
        fn(g.off + (long long)y * g.pitch + x0, cnt, ly, lx0);
    }
}

// Vectors of a tile, kStencilThreads threads: R rounds of one vector each.
template <typename T>
struct TileVec {
    static constexpr int VN = TileDim<T>::VN, VR = kTileW / VN, TOTAL = TileDim<T>::TH * VR;
    static constexpr int R = (TOTAL + kStencilThreads - 1) / kStencilThreads;
};

// First phase of a two-phase visit: load(d0, cnt) for every vector of the
// thread, into v; nothing waits for the loads here.  blockDim.x ==
// kStencilThreads.
template <typename T, typename FL, typename V>
__device__ __forceinline__ void tile_vec_load(const SliceGeom& g, const Item& it, FL load, V (&v)[TileVec<T>::R]) {
    using TV = TileVec<T>;
#pragma unroll
    for (int u = 0; u < TV::R; ++u) {
        const int q = threadIdx.x + u * kStencilThreads;
        const int ly = q / TV::VR, lx0 = (q - ly * TV::VR) * TV::VN;
        const int y = it.b + ly, x0 = it.a + lx0;
        if (q < TV::TOTAL && y < g.ny && x0 < g.nx)
            v[u] = load(g.off + (long long)y * g.pitch + x0, g.nx - x0 < TV::VN ? g.nx - x0 : TV::VN);
    }
}

// Second phase: store(d0, cnt, ly, lx0, loaded) for each vector loaded by
// tile_vec_load.
template <typename T, typename FS, typename V>
__device__ __forceinline__ void tile_vec_use(const SliceGeom& g, const Item& it, FS store,
                                             const V (&v)[TileVec<T>::R]) {
    using TV = TileVec<T>;
#pragma unroll
    for (int u = 0; u < TV::R; ++u) {
        const int q = threadIdx.x + u * kStencilThreads;
        const int ly = q / TV::VR, lx0 = (q - ly * TV::VR) * TV::VN;
        const int y = it.b + ly, x0 = it.a + lx0;
        if (q < TV::TOTAL && y < g.ny && x0 < g.nx)
            store(g.off + (long long)y * g.pitch + x0, g.nx - x0 < TV::VN ? g.nx - x0 : TV::VN, ly, lx0, v[u]);
    }
}

// As for_tile_vectors, in two phases: the loads of all rounds are in flight
// together.
template <typename T, typename FL, typename FS>
__device__ __forceinline__ void for_tile_vectors2(const SliceGeom& g, const Item& it, FL load, FS store) {
    using V = decltype(load(0LL, 0));
    V v[TileVec<T>::R];
    tile_vec_load<T>(g, it, load, v);
    tile_vec_use<T>(g, it, store, v);
}

template <typename T>
__device__ __forceinline__ Pack<T> ldv_n(const T* p, long long d, int cnt) {
    if (cnt == TileDim<T>::VN) return ldv(p, d);
    Pack<T> r;
#pragma unroll
    for (int e = 0; e < TileDim<T>::VN; ++e) r.v[e] = e < cnt ? p[d + e] : T(0);
    return r;
}
template <typename T>
__device__ __forceinline__ void stv_n(T* p, long long d, const Pack<T>& v, int cnt) {
    if (cnt == TileDim<T>::VN) {
        stv(p, d, v);
        return;
    }
#pragma unroll
    for (int e = 0; e < TileDim<T>::VN; ++e)
        if (e < cnt) p[d + e] = v.v[e];
}

// --------------------------------------------------------------------------
// K1: hard threshold (eq. sol_hv) + right-hand sides
// --------------------------------------------------------------------------

template <typename T, bool STATS>
__global__ void __launch_bounds__(kStencilThreads, 4) k_thr_rhs(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                             SliceState* S, Ptrs<T> P) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, SW = TileDim<T>::SW;
    __shared__ __align__(16) T sm[4][TileDim<T>::TH + 2][SW];
    __shared__ double red[9 * 32];
    __shared__ SliceGeom s_g;
    __shared__ SliceConst s_c;
    __shared__ SliceState s_st;
    const T* f1p = P.f[RECON_F_F1];
    const T* f2p = P.f[RECON_F_F2];
    const T* rhp = P.f[RECON_F_RHO];
    const T* zp = P.f[RECON_F_Z];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        if (!__ldg(&S[it.slice].active)) continue;
        stage_struct(&s_g, G + it.slice);
        stage_struct(&s_c, C + it.slice);
        stage_struct(&s_st, S + it.slice);
        __syncthreads();
        const SliceGeom& g = s_g;
        account(P.acct, KF_THR_RHS, tile_px<T>(g, it) * 10 * (long long)sizeof(T));
        load_tile<T, 4>(
            sm, g, it.a, it.b,
            [&](long long d) { return Vals<T, 4>{{f1p[d], f2p[d], rhp[d], zp[d]}}; },
            [&](long long d) { return PVals<T, 4>{{ldv(f1p, d), ldv(f2p, d), ldv(rhp, d), ldv(zp, d)}}; });
        __syncthreads();
        const SliceConst& c = s_c;
        const T thr = thr_of<T>(s_st);
        const T beta = Sc<T>::beta(s_st), beta_t = Sc<T>::beta_t(s_st);
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        // image domain: uL, uH = mu_hat(E_L), mu_hat(E_H).  Sinogram domain
        // (domain 1): uL, uH = t_1, t_2 and G1, G2 = A^T A f1, A^T A f2
        const bool sino = c.domain != 0;
        struct In {
            Pack<T> uL, uH, G1, G2;
        };
        auto load = [&](long long d, int cnt) {
            In x;
            x.uL = ldv_n(P.f[RECON_F_MUL], d, cnt);
            x.uH = ldv_n(P.f[RECON_F_MUH], d, cnt);
            if (sino) {
                x.G1 = ldv_n(P.f[RECON_F_A2], d, cnt);
                x.G2 = ldv_n(P.f[RECON_F_RHS_Z], d, cnt);
            }
            return x;
        };
        // thresholded divergence of map m at (ry, lx) of the tile (eq. sol_hv,
        // periodic forward differences; the statistics of the kept gradient)
        auto div_of = [&](int m, int ry, int lx, bool in) -> T {
            const T gc = sm[m][ry][lx];
            const T dx = sub_rn(sm[m][ry][lx + 1], gc);
            const T dy = sub_rn(sm[m][ry + 1][lx], gc);
            const T dxl = sub_rn(gc, sm[m][ry][lx - 1]);
            const T dyl = sub_rn(sm[m][ry + 1][lx - 1], sm[m][ry][lx - 1]);
            const T dxu = sub_rn(sm[m][ry - 1][lx + 1], sm[m][ry - 1][lx]);
            const T dyu = sub_rn(gc, sm[m][ry - 1][lx]);
            const bool k0 = keep_grad(dx, dy, thr);
            const bool kl = keep_grad(dxl, dyl, thr);
            const bool ku = keep_grad(dxu, dyu, thr);
            const T h0 = k0 ? dx : T(0), v0 = k0 ? dy : T(0);
            const T hl = kl ? dxl : T(0), vu = ku ? dyu : T(0);
            if (STATS && in) {
                if (!k0) acc[4] += (double)dx * dx + (double)dy * dy;
                acc[5 + m] += k0 ? 1.0 : 0.0;
            }
            return (hl - h0) + (vu - v0);
        };
        // pass A: f1, f2 (thresholds, right-hand sides, data and model terms)
        for_tile_vectors<T>(g, it, [&](long long d0, int cnt, int ly, int lx0) {
            const In x = load(d0, cnt);
            const Pack<T>&uL = x.uL, &uH = x.uH, &G1 = x.G1, &G2 = x.G2;
            Pack<T> o0, o1;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int lx = OFF + lx0 + e;   // column of this pixel in sm
                const int ry = ly + 1;
                const bool in = e < cnt;
                const T div0 = div_of(0, ry, lx, in), div1 = div_of(1, ry, lx, in);
                const T f1 = sm[0][ry][lx], f2 = sm[1][ry][lx], rho = sm[2][ry][lx], z = sm[3][ry][lx];
                const T M1 = rho * (kc<T>(c, KC_P1) * z + kc<T>(c, KC_PSI1));
                const T M2 = rho * (kc<T>(c, KC_P2) * z + kc<T>(c, KC_PSI2));
                const T b00 = kc<T>(c, KC_B00), b01 = kc<T>(c, KC_B01), b10 = kc<T>(c, KC_B10),
                        b11 = kc<T>(c, KC_B11), c12 = kc<T>(c, KC_C12);
                if (!sino) {
                    const T base1 = kc<T>(c, KC_A00) * uL.v[e] + kc<T>(c, KC_A01) * uH.v[e] + b00 * M1 + b01 * M2;
                    const T base2 = kc<T>(c, KC_A10) * uL.v[e] + kc<T>(c, KC_A11) * uH.v[e] + b10 * M1 + b11 * M2;
                    o0.v[e] = base1 - c12 * f2 + beta * div0;
                    o1.v[e] = (c.order ? base2 : base2 - c12 * f1) + beta * div1;
                } else {
                    // t_k - cross A^T A f_o / gamma + sum_j b_kj (M_j - f_o b_oj) + beta div
                    const T ag = kc<T>(c, KC_SINO_AG), bc = kc<T>(c, KC_SINO_BC);
                    o0.v[e] = uL.v[e] + b00 * M1 + b01 * M2 - ag * G2.v[e] - bc * f2 + beta * div0;
                    o1.v[e] = uH.v[e] + b10 * M1 + b11 * M2 - ag * G1.v[e] - bc * f1 + beta * div1;
                }
                if (STATS && in) {
                    const double dL = sino ? 0.0 : c.a00 * (double)f1 + c.a10 * (double)f2 - (double)uL.v[e];
                    const double dH = sino ? 0.0 : c.a01 * (double)f1 + c.a11 * (double)f2 - (double)uH.v[e];
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
            stv_n(P.f[RECON_F_RHS_F1], d0, o0, cnt);
            stv_n(P.f[RECON_F_RHS_F2], d0, o1, cnt);
        });
        // pass B: rho_e, z (thresholds, beta~-weighted divergences), from shared memory only
        for_tile_vectors<T>(g, it, [&](long long d0, int cnt, int ly, int lx0) {
            Pack<T> o2, o3;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int lx = OFF + lx0 + e, ry = ly + 1;
                const bool in = e < cnt;
                o2.v[e] = beta_t * div_of(2, ry, lx, in);
                o3.v[e] = beta_t * div_of(3, ry, lx, in);
            }
            stv_n(P.f[RECON_F_DIV_RHO], d0, o2, cnt);
            stv_n(P.f[RECON_F_DIV_Z], d0, o3, cnt);
        });
        if (STATS) {
            block_sum<9>(acc, red);
            double tot[9];
            if (item_reduce<9>(L, w, it.slice, acc, tot, red)) {
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
        if (!__ldg(&S[it.slice].active)) continue;
        const SliceGeom g = G[it.slice];
        const T c12 = T(C[it.slice].c12);
        for (int q = threadIdx.x; q < kTileW * TileH<T>::v; q += blockDim.x) {
            const int x = it.a + (q & (kTileW - 1)), y = it.b + q / kTileW;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            P.f[RECON_F_RHS_F2][d] -= c12 * P.f[RECON_F_F1][d];
        }
    }
}

// --------------------------------------------------------------------------
// FFT-diagonalised solve: rows (R2C, two real rows per complex FFT),
// columns (FFT, divide by c + beta K, inverse FFT), rows (C2R).
//
// Power-of-two sizes (FP32) take compile-time transforms whose first stage
// reads HBM and whose last stage writes it; other 7-smooth sizes take the
// runtime mixed-radix transform with a load phase and a store phase.
// --------------------------------------------------------------------------

// Sizes with compile-time transforms: powers of two 64 .. 1024 and the
// mixed sizes 320 (8 8 5), 384 (8 8 2 3), 448 (8 8 7).
__device__ __forceinline__ bool p2_fast(int n) {
    return n == 64 || n == 128 || n == 256 || n == 512 || n == 1024 || n == 320 || n == 384 || n == 448;
}

// Runs the statements with `constexpr int NN` set to n (one of p2_fast).
#define RECON_P2_DISPATCH(n, ...)                \
    switch (n) {                                 \
        case 64: {                               \
            constexpr int NN = 64;               \
            __VA_ARGS__;                         \
        } break;                                 \
        case 128: {                              \
            constexpr int NN = 128;              \
            __VA_ARGS__;                         \
        } break;                                 \
        case 256: {                              \
            constexpr int NN = 256;              \
            __VA_ARGS__;                         \
        } break;                                 \
        case 512: {                              \
            constexpr int NN = 512;              \
            __VA_ARGS__;                         \
        } break;                                 \
        case 320: {                              \
            constexpr int NN = 320;              \
            __VA_ARGS__;                         \
        } break;                                 \
        case 384: {                              \
            constexpr int NN = 384;              \
            __VA_ARGS__;                         \
        } break;                                 \
        case 448: {                              \
            constexpr int NN = 448;              \
            __VA_ARGS__;                         \
        } break;                                 \
        default: {                               \
            constexpr int NN = 1024;             \
            __VA_ARGS__;                         \
        } break;                                 \
    }

// Split the transforms of np row pairs (natural order in `res`) into the two
// half spectra of each pair: A = (Z_k + conj Z_-k)/2, B = (Z_k - conj Z_-k)/(2i).
// ---- asynchronous tile copies (cp.async: global -> shared, no registers) ----

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// 16 bytes; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// one element of B = 4 or 8 bytes
template <int B>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ void rows_to_half_spectra(const cplx<T>* res, int ld, int N, int nh, int np, int rows,
                                                     cplx<T>* spr, int cpitch) {
    const DivMod dh(nh);
    for (int q = threadIdx.x; q < np * nh; q += blockDim.x) {
        const int b = dh.div(q), k = q - b * nh;
        const cplx<T> zk = res[b * ld + pad8(k)];
        const cplx<T> zc = res[b * ld + pad8(k == 0 ? 0 : N - k)];
        const long long e0 = (long long)(2 * b) * cpitch + k;
        spr[e0] = {T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
        if (2 * b + 1 < rows) spr[e0 + cpitch] = {T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
    }
}

// Element n of the complex sequence A + iB whose inverse transform gives the
// real rows of the half spectra ra (real part) and rb (imaginary part; null
// for none); the upper half follows from Hermitian symmetry.
template <typename T>
__device__ __forceinline__ cplx<T> row_pair_from_half_spectra(const cplx<T>* ra, const cplx<T>* rb, int N, int nh,
                                                             int n) {
    const bool upper = n >= nh;
    const int k = upper ? N - n : n;
    cplx<T> a = ra[k], c = {T(0), T(0)};
    if (rb) c = rb[k];
    if (upper) {
        a.y = -a.y;
        c.y = -c.y;
    }
    return {a.x - c.y, a.y + c.x};
}

// Item: rows 2*it.a .. of one slice, it.b pairs; two real rows per complex FFT.
template <typename T>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) k_rows_fwd(ItemList L, const SliceGeom* G, const SliceState* S,
                                                           Ptrs<T> P, FftJobs J, const cplx<T>* twpool, int half) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf2 = buf + half;
    const int total = L.n_items * J.n;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int job = w / L.n_items, item = w - job * L.n_items;
        const Item it = L.items[item];
        if (!__ldg(&S[it.slice].active) || (J.coef[job] >= 3 && __ldg(&S[it.slice].cg_done))) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.nx, pair0 = it.a, np = it.b, ld = padded_len(N);
        const int rows = (g.ny - 2 * pair0 < 2 * np) ? g.ny - 2 * pair0 : 2 * np;
        account(P.acct, KF_ROWS_FWD, (long long)rows * (N * (long long)sizeof(T) + g.nh * 2 * (long long)sizeof(T)));
        const T* inr = P.f[J.in[job]] + g.off + (long long)(2 * pair0) * g.pitch;
        const cplx<T>* tw = twpool + g.twx;
        const cplx<T>* res;
        auto elem = [&](int b, int n) -> cplx<T> {
            const long long d = (long long)(2 * b) * g.pitch + n;
            return {inr[d], 2 * b + 1 < rows ? inr[d + g.pitch] : T(0)};
        };
        bool fast = false;
        if constexpr (std::is_same<T, float>::value) fast = p2_fast(N);
        if (fast) {
            // the item's rows land in buf2 first, all copies in flight at once (rows x N reals, which fit:
            // the item's transforms take (np + 1) padded sequences of N complex slots)
            T* stg = reinterpret_cast<T*>(buf2);
            const int nv = N / 4;   // 16-byte vectors per row (N >= 64)
            for (int q = threadIdx.x; q < rows * nv; q += blockDim.x) {
                const int rr = q / nv, v4 = q - rr * nv;
                cp_async16(stg + rr * N + 4 * v4, inr + (long long)rr * g.pitch + 4 * v4);
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            auto selem = [&](int b, int n) -> cplx<T> {
                return {stg[2 * b * N + n], 2 * b + 1 < rows ? stg[(2 * b + 1) * N + n] : T(0)};
            };
            RECON_P2_DISPATCH(N, p2_stage<T, NN, 0, -1, false, 1>(np, tw + NN, fn_load<T>(selem), SmemSeq<T>{buf, ld});
                              __syncthreads();
                              res = p2_smem_stages<T, NN, -1, 1, P2Plan<NN>::S - 1>(buf, buf2, ld, np, tw + NN));
        } else {
            // four elements per thread per round, loads issued before use
            const DivMod dN(N);
            const int total_q = np * N;
            for (int q0 = threadIdx.x; q0 < total_q; q0 += 4 * blockDim.x) {
                cplx<T> v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q < total_q) {
                        const int b = dN.div(q);
                        v[u] = elem(b, q - b * N);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q < total_q) {
                        const int b = dN.div(q);
                        buf[b * ld + pad8(q - b * N)] = v[u];
                    }
                }
            }
            __syncthreads();
            res = fft_batch<T>(buf, buf2, N, g.plan_x, np, ld, tw, -1);
        }
        rows_to_half_spectra(res, ld, N, g.nh, np, rows,
                             P.s[J.spec[job]] + g.coff + (long long)(2 * pair0) * g.cpitch, g.cpitch);
        __syncthreads();
    }
}

// Column item, power-of-two N: forward transform along y (first stage read
// straight from the spectrum, column-fastest), the spectral divide folded into
// the last forward stage, inverse transform with the last stage written
// straight back.  With RY, adds sum_k w_kx |X_k|^2 / (n m_k) over the item to
// `acc` (the item's share of u.(m(F))^-1 u by Parseval; w = 1 on the columns
// kx = 0 and kx = nx/2, which stand for themselves, 2 on the others, which
// also stand for their conjugate partners outside the half spectrum).
template <typename T, int N, bool RY>
__device__ __forceinline__ void cols_item_p2(cplx<T>* spc, int cpitch, int nc, int col0, int nx, cplx<T>* buf0,
                                             cplx<T>* buf1, const cplx<T>* tw, const T* symx, const T* symy, T cst,
                                             T bet, T inv_n, T& acc) {
    constexpr int S = P2Plan<N>::S;
    constexpr int E = FftBudget<T>::E / N;
    constexpr int CB = E > 16 ? 16 : (E < 1 ? 1 : E);
    const int ld = col_ld(N);
    // the item's columns land in buf1 first, row-major (N rows of CB slots), all copies in flight at
    // once.  With CB and col0 even (the power-of-two sizes) a copy moves a pair of columns, 16-byte
    // aligned on both sides (the spectrum's offsets and pitch are multiples of 16 slots), and the last
    // pair of an odd count reads one padding column of the row (nh odd, so the pitch exceeds it).
    // Otherwise (CB = 9 or col0 odd for N = 448) one column per copy.
    if (((CB | col0) & 1) == 0) {
        const int nv = (nc + 1) / 2;
        for (int q = threadIdx.x; q < N * nv; q += blockDim.x) {
            const int y = q / nv, v2 = q - y * nv;
            cp_async16(buf1 + y * CB + 2 * v2, spc + (long long)y * cpitch + 2 * v2);
        }
    } else {
        for (int q = threadIdx.x; q < N * nc; q += blockDim.x) {
            const int y = q / nc, b = q - y * nc;
            cp_async_elem<sizeof(cplx<T>)>(buf1 + y * CB + b, spc + (long long)y * cpitch + b);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    auto sload = [&](int b, int y) -> cplx<T> { return buf1[y * CB + b]; };
    p2_stage<T, N, 0, -1, true, CB>(nc, tw + N, fn_load<T>(sload), SmemSeq<T>{buf0, ld});
    __syncthreads();
    cplx<T>* cur = p2_smem_stages<T, N, -1, 1, S - 2>(buf0, buf1, ld, nc, tw + N);
    cplx<T>* oth = cur == buf0 ? buf1 : buf0;
    // |F dx|^2 + |F dy|^2 = 4 sin^2(pi kx / nx) + 4 sin^2(pi ky / ny)
    auto divide = [&](int b, int ky, cplx<T> v) {
        const T sc = inv_n / (cst + bet * (symx[col0 + b] + symy[ky]));
        if (RY) {
            const int kx = col0 + b;
            const T wgt = (kx == 0 || 2 * kx == nx) ? T(1) : T(2);
            acc = fma(wgt * sc, v.x * v.x + v.y * v.y, acc);
        }
        oth[b * ld + pad8(ky)] = {v.x * sc, v.y * sc};
    };
    p2_stage<T, N, S - 1, -1, false, 1>(nc, tw + N, SmemSeq<T>{cur, ld}, fn_store<T>(divide));
    __syncthreads();
    cur = p2_smem_stages<T, N, +1, 0, S - 2>(oth, cur, ld, nc, tw + N);
    auto gstore = [&](int b, int y, cplx<T> v) { spc[(long long)y * cpitch + b] = v; };
    p2_stage<T, N, S - 1, +1, true, CB>(nc, tw + N, SmemSeq<T>{cur, ld}, fn_store<T>(gstore));
    __syncthreads();
}

// Column pass.  Kinds 0, 1, 2 divide by c_f1 + beta K, c_f2 + beta K,
// 1 + beta~ K (the f1, f2 and rho_e solves); kind 3 divides by
// abar^2 + beta~ K (the PCG preconditioner) and also reduces r.y of the PCG
// step over the slice, which sets beta_cg = (r.y)/(r.y)_old.
template <typename T>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) k_cols(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                       SliceState* S, Ptrs<T> P, FftJobs J,
                                                       const cplx<T>* twpool, int half, int rev = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf1 = buf0 + half;
    __shared__ double red[32];
    const int total = L.n_items * J.n;
    for (int w0 = blockIdx.x; w0 < total; w0 += gridDim.x) {
        const int w = rev ? total - 1 - w0 : w0;   // reversed order: see op_solve_z
        const int job = w / L.n_items, item = w - job * L.n_items;
        const Item it = L.items[item];
        const int kind = J.coef[job];
        const SliceState* st = S + it.slice;
        if (!__ldg(&st->active) || (kind >= 3 && __ldg(&st->cg_done))) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.ny, col0 = it.a, nc = it.b, ld = col_ld(N);
        account(P.acct, kind == 3 ? KF_COLS_PRE : (kind > 3 ? KF_FCG : KF_COLS),
                (long long)nc * N * 4 * (long long)sizeof(T));
        cplx<T>* sp = P.s[J.spec[job]];
        const cplx<T>* tw = twpool + g.twy;
        T cst, bet;
        switch (kind) {
            case 0: cst = kc<T>(C[it.slice], KC_CF1); bet = Sc<T>::beta(*st); break;
            case 1: cst = kc<T>(C[it.slice], KC_CF2); bet = Sc<T>::beta(*st); break;
            case 2: cst = T(1); bet = Sc<T>::beta_t(*st); break;
            case 3: cst = Sc<T>::abar2(*st); bet = Sc<T>::beta_t(*st); break;
            case 4: cst = kc<T>(C[it.slice], KC_SINO_D0); bet = Sc<T>::beta(*st); break;
            default: cst = kc<T>(C[it.slice], KC_SINO_D1); bet = Sc<T>::beta(*st); break;
        }
        const T inv_n = inv_n_of<T>(g);
        const T* symx = P.sym + g.symx;
        const T* symy = P.sym + g.symy;
        T accT = T(0);
        bool fast = false;
        if constexpr (std::is_same<T, float>::value) fast = p2_fast(N);
        if (fast) {
            cplx<T>* spc = sp + g.coff + col0;
            if (kind >= 3) {
                RECON_P2_DISPATCH(N, cols_item_p2<T, NN, true>(spc, g.cpitch, nc, col0, g.nx, buf0, buf1, tw, symx,
                                                               symy, cst, bet, inv_n, accT));
            } else {
                RECON_P2_DISPATCH(N, cols_item_p2<T, NN, false>(spc, g.cpitch, nc, col0, g.nx, buf0, buf1, tw, symx,
                                                                symy, cst, bet, inv_n, accT));
            }
        } else {
            {
                const DivMod dc(nc);
                const int total_q = nc * N;
                for (int q0 = threadIdx.x; q0 < total_q; q0 += 4 * blockDim.x) {
                    cplx<T> v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u * blockDim.x;
                        if (q < total_q) {
                            const int y = dc.div(q), cc = q - y * nc;
                            v[u] = sp[g.coff + (long long)y * g.cpitch + col0 + cc];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u * blockDim.x;
                        if (q < total_q) {
                            const int y = dc.div(q), cc = q - y * nc;
                            buf0[cc * ld + pad8(y)] = v[u];
                        }
                    }
                }
            }
            __syncthreads();
            // forward FFT along y, spectral divide, inverse FFT along y (one
            // inlined transform, run twice)
            cplx<T>* buf = buf0;
            for (int pass = 0; pass < 2; ++pass) {
                buf = fft_batch<T>(buf, buf == buf0 ? buf1 : buf0, N, g.plan_y, nc, ld, tw, pass ? +1 : -1);
                if (pass) break;
                const DivMod dN(N);
                for (int q = threadIdx.x; q < nc * N; q += blockDim.x) {
                    const int cc = dN.div(q), ky = q - cc * N;
                    // |F dx|^2 + |F dy|^2 = 4 sin^2(pi kx / nx) + 4 sin^2(pi ky / ny)
                    const T sc = inv_n / (cst + bet * (symx[col0 + cc] + symy[ky]));
                    cplx<T> v = buf[cc * ld + pad8(ky)];
                    if (kind >= 3) {
                        const int kx = col0 + cc;
                        const T wgt = (kx == 0 || 2 * kx == g.nx) ? T(1) : T(2);
                        accT = fma(wgt * sc, v.x * v.x + v.y * v.y, accT);
                    }
                    buf[cc * ld + pad8(ky)] = {v.x * sc, v.y * sc};
                }
                __syncthreads();
            }
            {
                const DivMod dc(nc);
                for (int q = threadIdx.x; q < nc * N; q += blockDim.x) {
                    const int y = dc.div(q), cc = q - y * nc;
                    sp[g.coff + (long long)y * g.cpitch + col0 + cc] = buf[cc * ld + pad8(y)];
                }
            }
            __syncthreads();
        }
        if (kind >= 3) {
            const T part[1] = {accT};
            double acc[1];
            block_sum_t<T, 1>(part, acc, red);
            double tot[1];
            if (item_reduce<1>(L, item, it.slice, acc, tot, red)) {
                SliceState& so = S[it.slice];
                set_betacg(so, (so.cg_it == 0) ? 0.0 : tot[0] / so.ry);
                so.ry = tot[0];
            }
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) k_rows_inv(ItemList L, const SliceGeom* G, const SliceState* S,
                                                           Ptrs<T> P, FftJobs J, const cplx<T>* twpool, int half) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf2 = buf + half;
    const int total = L.n_items * J.n;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int job = w / L.n_items, item = w - job * L.n_items;
        const Item it = L.items[item];
        if (!__ldg(&S[it.slice].active) || (J.coef[job] >= 3 && __ldg(&S[it.slice].cg_done))) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.nx, pair0 = it.a, np = it.b, ld = padded_len(N);
        const int rows = (g.ny - 2 * pair0 < 2 * np) ? g.ny - 2 * pair0 : 2 * np;
        account(P.acct, KF_ROWS_INV, (long long)rows * (N * (long long)sizeof(T) + g.nh * 2 * (long long)sizeof(T)));
        const cplx<T>* spr = P.s[J.spec[job]] + g.coff + (long long)(2 * pair0) * g.cpitch;
        T* outr = P.f[J.out[job]] + g.off + (long long)(2 * pair0) * g.pitch;
        const cplx<T>* tw = twpool + g.twx;
        auto elem = [&](int b, int n) -> cplx<T> {
            const cplx<T>* ra = spr + (long long)(2 * b) * g.cpitch;
            return row_pair_from_half_spectra<T>(ra, 2 * b + 1 < rows ? ra + g.cpitch : nullptr, N, g.nh, n);
        };
        auto put = [&](int b, int n, cplx<T> v) {
            const long long d = (long long)(2 * b) * g.pitch + n;
            outr[d] = v.x;
            if (2 * b + 1 < rows) outr[d + g.pitch] = v.y;
        };
        bool fast = false;
        if constexpr (std::is_same<T, float>::value) fast = p2_fast(N);
        if (fast) {
            // the item's half-spectrum rows land in buf2 first (rows x sw complex, sw = nh rounded up to
            // even, which fits beside the (np + 1) padded sequences of the item's transforms)
            cplx<T>* stg = buf2;
            const int sw = (g.nh + 1) & ~1, nv = sw / 2;
            for (int q = threadIdx.x; q < rows * nv; q += blockDim.x) {
                const int rr = q / nv, v2 = q - rr * nv;
                cp_async16(stg + rr * sw + 2 * v2, spr + (long long)rr * g.cpitch + 2 * v2);
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            auto selem = [&](int b, int n) -> cplx<T> {
                const cplx<T>* ra = stg + 2 * b * sw;
                return row_pair_from_half_spectra<T>(ra, 2 * b + 1 < rows ? ra + sw : nullptr, N, g.nh, n);
            };
            RECON_P2_DISPATCH(N, p2_stage<T, NN, 0, +1, false, 1>(np, tw + NN, fn_load<T>(selem), SmemSeq<T>{buf, ld});
                              __syncthreads();
                              cplx<T>* cur = p2_smem_stages<T, NN, +1, 1, P2Plan<NN>::S - 2>(buf, buf2, ld, np, tw + NN);
                              p2_stage<T, NN, P2Plan<NN>::S - 1, +1, false, 1>(np, tw + NN, SmemSeq<T>{cur, ld},
                                                                              fn_store<T>(put)));
        } else {
            const DivMod dN(N);
            const int total_q = np * N;
            for (int q0 = threadIdx.x; q0 < total_q; q0 += 4 * blockDim.x) {
                cplx<T> v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q < total_q) {
                        const int b = dN.div(q);
                        v[u] = elem(b, q - b * N);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q < total_q) {
                        const int b = dN.div(q);
                        buf[b * ld + pad8(q - b * N)] = v[u];
                    }
                }
            }
            __syncthreads();
            const cplx<T>* res = fft_batch<T>(buf, buf2, N, g.plan_x, np, ld, tw, +1);
            for (int q = threadIdx.x; q < total_q; q += blockDim.x) {
                const int b = dN.div(q), n = q - b * N;
                put(b, n, res[b * ld + pad8(n)]);
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// PCG of the Z^m step (Alg. 1): M z = ab + beta~ div(h, v) with
// M = diag(a^2) + beta~ (dx'dx + dy'dy), preconditioner
// D^-1/2 (abar^2 + beta~ L)^-1 D^-1/2, D = diag((a^2 + 4 beta~)/(abar^2 + 4 beta~)).
// A step takes three passes over row-pair items and column items:
//   k_pcg_fwd  z += alpha p, r -= alpha q, r.r and the convergence test;
//              u = D^-1/2 r; row transforms of u -> half spectrum
//   k_cols     column transforms, r.y = u.(abar^2 + beta~ L)^-1 u taken in
//              the spectral domain, divide, inverse columns -> beta_cg
//   k_pcg_inv  inverse row transforms -> x = (abar^2 + beta~ L)^-1 u on the
//              item's rows and the rows just above and below it;
//              p = D^-1/2 x + beta_cg p_old; q = M p; p.q -> alpha
// --------------------------------------------------------------------------

// Stage-0 source of the forward row transform of a PCG step: element n of
// rows 2b and 2b+1 of the item gets z += alpha p and r -= alpha q (UPD), adds
// r^2 to `acc`, and enters the transform as u = D^-1/2 r.  The loads of four
// legs are issued before any store.
template <typename T, bool UPD>
struct PcgFwdLoad {
    T* z;
    T* r;
    const T* p;
    const T* q;
    const T* a2;
    int pitch, rows;
    T al, rnum, b4;
    T& acc;

    __device__ __forceinline__ cplx<T> one(int b, int n) const {
        T u[2] = {T(0), T(0)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && 2 * b + 1 >= rows) break;
            const long long d = (long long)(2 * b + h) * pitch + n;
            T rv = r[d];
            const T w = a2[d];
            if (UPD) {
                z[d] = fma(al, p[d], z[d]);
                rv = fma(-al, q[d], rv);
                r[d] = rv;
                acc = fma(rv, rv, acc);
            }
            u[h] = rv * dscale(rnum, w, b4);
        }
        return {u[0], u[1]};
    }

    template <int R, int NBF>
    __device__ __forceinline__ void load_legs(int b, int j, cplx<T>* v) const {
        constexpr int G4 = R < 4 ? R : 4;
        static_assert(R % G4 == 0, "first-stage radix of the row transforms is 2, 4 or 8");
        const long long d0 = (long long)(2 * b) * pitch + j;
        const bool has1 = 2 * b + 1 < rows;
#pragma unroll
        for (int g0 = 0; g0 < R; g0 += G4) {
            T rv[2][G4], wv[2][G4], zv[2][G4], pv[2][G4], qv[2][G4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int u = 0; u < G4; ++u) {
                    const long long d = d0 + h * pitch + (g0 + u) * NBF;
                    const bool ok = h == 0 || has1;
                    rv[h][u] = ok ? r[d] : T(0);
                    wv[h][u] = ok ? a2[d] : T(0);
                    if (UPD) {
                        zv[h][u] = ok ? z[d] : T(0);
                        pv[h][u] = ok ? p[d] : T(0);
                        qv[h][u] = ok ? q[d] : T(0);
                    }
                }
#pragma unroll
            for (int u = 0; u < G4; ++u) {
                T uo[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    T rn = rv[h][u];
                    if (UPD && (h == 0 || has1)) {
                        const long long d = d0 + h * pitch + (g0 + u) * NBF;
                        z[d] = fma(al, pv[h][u], zv[h][u]);
                        rn = fma(-al, qv[h][u], rn);
                        r[d] = rn;
                        acc = fma(rn, rn, acc);
                    }
                    uo[h] = (h == 0 || has1) ? rn * dscale(rnum, wv[h][u], b4) : T(0);
                }
                v[g0 + u] = {uo[0], uo[1]};
            }
        }
    }
};

// UPD = false: the first step of the solve (r from k_cg_init, no update).
template <typename T, bool UPD>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) k_pcg_fwd(ItemList L, const SliceGeom* G,
                                                                        const SliceConst* C, SliceState* S, Ptrs<T> P,
                                                                        const cplx<T>* twpool, int half, int par,
                                                                        int* pending, int rev = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf2 = buf + half;
    __shared__ double red[32];
    for (int w0 = blockIdx.x; w0 < L.n_items; w0 += gridDim.x) {
        const int item = rev ? L.n_items - 1 - w0 : w0;
        const Item it = L.items[item];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.nx, np = it.b, ld = padded_len(N), r0 = 2 * it.a;
        const int rows = (g.ny - r0 < 2 * np) ? g.ny - r0 : 2 * np;
        account(P.acct, KF_PCG_FWD,
                (long long)rows * ((UPD ? 7 : 2) * N * (long long)sizeof(T) + g.nh * 2 * (long long)sizeof(T)));
        const long long d0 = g.off + (long long)r0 * g.pitch;
        T acc = T(0);
        const PcgFwdLoad<T, UPD> src{P.f[RECON_F_Z] + d0,
                                     P.f[RECON_F_CG_R] + d0,
                                     P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1] + d0,
                                     P.f[RECON_F_CG_Q] + d0,
                                     P.f[RECON_F_A2] + d0,
                                     g.pitch,
                                     rows,
                                     UPD ? Sc<T>::alpha(*sp) : T(0),
                                     Sc<T>::rnum(*sp),
                                     Sc<T>::b4(*sp),
                                     acc};
        const cplx<T>* tw = twpool + g.twx;
        const cplx<T>* res;
        bool fast = false;
        if constexpr (std::is_same<T, float>::value) fast = p2_fast(N);
        if (fast) {
            RECON_P2_DISPATCH(N, p2_stage<T, NN, 0, -1, false, 1>(np, tw + NN, src, SmemSeq<T>{buf, ld});
                              __syncthreads();
                              res = p2_smem_stages<T, NN, -1, 1, P2Plan<NN>::S - 1>(buf, buf2, ld, np, tw + NN));
        } else {
            const DivMod dN(N);
            for (int q = threadIdx.x; q < np * N; q += blockDim.x) {
                const int b = dN.div(q), n = q - b * N;
                buf[b * ld + pad8(n)] = src.one(b, n);
            }
            __syncthreads();
            res = fft_batch<T>(buf, buf2, N, g.plan_x, np, ld, tw, -1);
        }
        rows_to_half_spectra(res, ld, N, g.nh, np, rows, P.s[0] + g.coff + (long long)r0 * g.cpitch, g.cpitch);
        if (UPD) {
            const T part[1] = {acc};
            double a[1];
            block_sum_t<T, 1>(part, a, red);
            double tot[1];
            if (item_reduce<1>(L, item, it.slice, a, tot, red)) {
                SliceState& so = S[it.slice];
                const SliceConst& c = C[it.slice];
                so.rr = tot[0];
                so.cg_it += 1;
                const bool conv = !(tot[0] > c.cg_tol * c.cg_tol * so.bb);
                if (conv || so.cg_it >= c.cg_max) {
                    so.cg_done = 1;
                    atomicSub(pending, 1);
                    atomicMax(pending + 1, so.cg_it);
                }
            }
        }
        __syncthreads();
    }
}

// Relative row i in [-1, rows] of a k_pcg_inv item -> (sequence, component):
// rows 0 .. rows-1 are pairs 0 .. np-1; row -1 (above) and row `rows`
// (below) form sequence np.
__device__ __forceinline__ int pcg_row_slot(int i, int rows, int np, int ld) {
    int b, comp;
    if (i < 0) {
        b = np;
        comp = 0;
    } else if (i >= rows) {
        b = np;
        comp = 1;
    } else {
        b = i >> 1;
        comp = i & 1;
    }
    return 2 * b * ld + comp;   // in scalars; add 2 * pad8(n)
}

// Tail of a k_pcg_inv item for a power-of-two row length N (FP32), four
// pixels per task with 16-byte loads and stores: p = D^-1/2 x + beta_cg p_old
// on rows -1 .. rows in place (x in `rx`, interleaved as the transforms left
// it), a^2 of the item's rows staged in `a2s`, then q = M p on the item's
// rows; returns this thread's share of p.q.
template <int N>
__device__ __forceinline__ float pcg_inv_tail_p2(float* rx, float* a2s, int ld, int np, int rows, int r0, int up,
                                                 int dn, long long off, int pitch, const float* __restrict__ a2,
                                                 const float* __restrict__ pold, float* __restrict__ pnew,
                                                 float* __restrict__ qo, bool first, float bc, float rnum, float b4,
                                                 float bt) {
    constexpr int NV = N / 4;
    {
        const int total = (rows + 2) * NV;
        for (int t0 = threadIdx.x; t0 < total; t0 += 4 * blockDim.x) {
            float4 wv[4], pv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u * blockDim.x;
                wv[u] = pv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t < total) {
                    const int i = t / NV - 1, n0 = (t % NV) * 4;
                    const int grow = i < 0 ? up : (i >= rows ? dn : r0 + i);
                    const long long d = off + (long long)grow * pitch + n0;
                    wv[u] = *reinterpret_cast<const float4*>(a2 + d);
                    if (!first) pv[u] = *reinterpret_cast<const float4*>(pold + d);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u * blockDim.x;
                if (t < total) {
                    const int i = t / NV - 1, n0 = (t % NV) * 4;
                    float* px = rx + pcg_row_slot(i, rows, np, ld) + 2 * pad8(n0);   // n0 % 4 == 0: legs at +2e
                    px[0] = fmaf(bc, pv[u].x, px[0] * dscale(rnum, wv[u].x, b4));
                    px[2] = fmaf(bc, pv[u].y, px[2] * dscale(rnum, wv[u].y, b4));
                    px[4] = fmaf(bc, pv[u].z, px[4] * dscale(rnum, wv[u].z, b4));
                    px[6] = fmaf(bc, pv[u].w, px[6] * dscale(rnum, wv[u].w, b4));
                    if (i >= 0 && i < rows) *reinterpret_cast<float4*>(a2s + i * N + n0) = wv[u];
                }
            }
        }
    }
    __syncthreads();
    float acc = 0.f;
    const int total = rows * NV;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int i = t / NV, n0 = (t % NV) * 4;
        const float* row = rx + pcg_row_slot(i, rows, np, ld);
        const float* rup = rx + pcg_row_slot(i - 1, rows, np, ld);
        const float* rdn = rx + pcg_row_slot(i + 1, rows, np, ld);
        const int o = 2 * pad8(n0);
        const float c[4] = {row[o], row[o + 2], row[o + 4], row[o + 6]};
        const float lf = row[2 * pad8(n0 == 0 ? N - 1 : n0 - 1)];
        const float rt = row[2 * pad8(n0 + 4 == N ? 0 : n0 + 4)];
        const float4 w4 = *reinterpret_cast<const float4*>(a2s + i * N + n0);
        const float w[4] = {w4.x, w4.y, w4.z, w4.w};
        float q[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float l = e == 0 ? lf : c[e - 1];
            const float r = e == 3 ? rt : c[e + 1];
            const float lp = (4.f * c[e] - l - r) - (rup[o + 2 * e] + rdn[o + 2 * e]);
            q[e] = w[e] * c[e] + bt * lp;
            acc = fmaf(c[e], q[e], acc);
        }
        const long long d = off + (long long)(r0 + i) * pitch + n0;
        *reinterpret_cast<float4*>(pnew + d) = make_float4(c[0], c[1], c[2], c[3]);
        *reinterpret_cast<float4*>(qo + d) = make_float4(q[0], q[1], q[2], q[3]);
    }
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) k_pcg_inv(ItemList L, const SliceGeom* G, SliceState* S,
                                                                        Ptrs<T> P, const cplx<T>* twpool, int half,
                                                                        int par, int rev = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf2 = buf + half;
    __shared__ double red[32];
    const T* pold = P.f[par ? RECON_F_CG_P1 : RECON_F_CG_P0];
    T* pnew = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    const T* a2 = P.f[RECON_F_A2];
    T* qo = P.f[RECON_F_CG_Q];
    for (int w0 = blockIdx.x; w0 < L.n_items; w0 += gridDim.x) {
        const int item = rev ? L.n_items - 1 - w0 : w0;
        const Item it = L.items[item];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const SliceGeom g = G[it.slice];
        const int N = g.nx, np = it.b, ld = padded_len(N), r0 = 2 * it.a;
        const int rows = (g.ny - r0 < 2 * np) ? g.ny - r0 : 2 * np;
        const int up = wrap(r0 - 1, g.ny), dn = wrap(r0 + rows, g.ny);
        account(P.acct, KF_PCG_INV,
                (long long)rows * (4 * N * (long long)sizeof(T) + g.nh * 2 * (long long)sizeof(T)));
        const cplx<T>* s0 = P.s[0] + g.coff;
        auto elem = [&](int b, int n) -> cplx<T> {
            const cplx<T>* ra;
            const cplx<T>* rb;
            if (b < np) {
                ra = s0 + (long long)(r0 + 2 * b) * g.cpitch;
                rb = 2 * b + 1 < rows ? ra + g.cpitch : nullptr;
            } else {
                ra = s0 + (long long)up * g.cpitch;
                rb = s0 + (long long)dn * g.cpitch;
            }
            return row_pair_from_half_spectra<T>(ra, rb, N, g.nh, n);
        };
        const cplx<T>* tw = twpool + g.twx;
        cplx<T>* res;
        bool fast = false;
        if constexpr (std::is_same<T, float>::value) fast = p2_fast(N);
        if (fast) {
            RECON_P2_DISPATCH(N, p2_stage<T, NN, 0, +1, false, 1>(np + 1, tw + NN, fn_load<T>(elem), SmemSeq<T>{buf, ld});
                              __syncthreads();
                              res = p2_smem_stages<T, NN, +1, 1, P2Plan<NN>::S - 1>(buf, buf2, ld, np + 1, tw + NN));
        } else {
            const DivMod dN(N);
            for (int q = threadIdx.x; q < (np + 1) * N; q += blockDim.x) {
                const int b = dN.div(q), n = q - b * N;
                buf[b * ld + pad8(n)] = elem(b, n);
            }
            __syncthreads();
            res = fft_batch<T>(buf, buf2, N, g.plan_x, np + 1, ld, tw, +1);
        }
        T* rx = reinterpret_cast<T*>(res);
        T* a2s = reinterpret_cast<T*>(res == buf ? buf2 : buf);   // a^2 of the interior rows
        const bool first = __ldg(&sp->cg_it) == 0;
        const T bc = first ? T(0) : Sc<T>::betacg(*sp);
        const T rnum = Sc<T>::rnum(*sp);
        const T b4 = Sc<T>::b4(*sp);
        const T bt = Sc<T>::beta_t(*sp);
        if constexpr (std::is_same<T, float>::value) {
            if (fast) {
                T acc = T(0);
                RECON_P2_DISPATCH(N, acc = pcg_inv_tail_p2<NN>(rx, a2s, ld, np, rows, r0, up, dn, g.off, g.pitch, a2,
                                                               pold, pnew, qo, first, bc, rnum, b4, bt));
                const T part[1] = {acc};
                double a[1];
                block_sum_t<T, 1>(part, a, red);
                double tot[1];
                if (item_reduce<1>(L, item, it.slice, a, tot, red)) {
                    SliceState& so = S[it.slice];
                    so.pq = tot[0];
                    set_alpha(so, tot[0] > 0.0 ? so.ry / tot[0] : 0.0);
                }
                __syncthreads();
                continue;
            }
        }
        const DivMod dN(N);
        // p = D^-1/2 x + beta_cg p_old on rows -1 .. rows, in place; four
        // elements per thread per round, loads issued before use
        {
            const int total_q = (rows + 2) * N;
            for (int q0 = threadIdx.x; q0 < total_q; q0 += 4 * blockDim.x) {
                T wv[4], pv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * blockDim.x;
                    wv[u] = pv[u] = T(0);
                    if (q < total_q) {
                        const int i = dN.div(q) - 1, n = q - (i + 1) * N;
                        const int grow = i < 0 ? up : (i >= rows ? dn : r0 + i);
                        const long long d = g.off + (long long)grow * g.pitch + n;
                        wv[u] = a2[d];
                        if (!first) pv[u] = pold[d];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q < total_q) {
                        const int i = dN.div(q) - 1, n = q - (i + 1) * N;
                        T* px = rx + pcg_row_slot(i, rows, np, ld) + 2 * pad8(n);
                        *px = fma(bc, pv[u], *px * dscale(rnum, wv[u], b4));
                        if (i >= 0 && i < rows) a2s[i * N + n] = wv[u];
                    }
                }
            }
        }
        __syncthreads();
        // q = a^2 p + beta~ (4p - p_left - p_right - p_up - p_down), p.q
        T acc = T(0);
        for (int q = threadIdx.x; q < rows * N; q += blockDim.x) {
            const int i = dN.div(q), n = q - i * N;
            const T* row = rx + pcg_row_slot(i, rows, np, ld);
            const T c = row[2 * pad8(n)];
            const T l = row[2 * pad8(n == 0 ? N - 1 : n - 1)];
            const T rr = row[2 * pad8(n == N - 1 ? 0 : n + 1)];
            const T u = rx[pcg_row_slot(i - 1, rows, np, ld) + 2 * pad8(n)];
            const T dw = rx[pcg_row_slot(i + 1, rows, np, ld) + 2 * pad8(n)];
            const T lp = (T(4) * c - l - rr) - (u + dw);
            const T qq = a2s[i * N + n] * c + bt * lp;
            const long long d = g.off + (long long)(r0 + i) * g.pitch + n;
            pnew[d] = c;
            qo[d] = qq;
            acc = fma(c, qq, acc);
        }
        const T part[1] = {acc};
        double a[1];
        block_sum_t<T, 1>(part, a, red);
        double tot[1];
        if (item_reduce<1>(L, item, it.slice, a, tot, red)) {
            SliceState& so = S[it.slice];
            so.pq = tot[0];
            set_alpha(so, tot[0] > 0.0 ? so.ry / tot[0] : 0.0);
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
    constexpr int VN = TileDim<T>::VN;
    __shared__ SliceGeom s_g;
    __shared__ SliceConst s_c;
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        if (!__ldg(&S[it.slice].active)) continue;
        stage_struct(&s_g, G + it.slice);
        stage_struct(&s_c, C + it.slice);
        __syncthreads();
        const SliceGeom& g = s_g;
        const SliceConst& c = s_c;
        account(P.acct, KF_SYNTH, tile_px<T>(g, it) * 7 * (long long)sizeof(T));
        const T b00 = kc<T>(c, KC_B00), b10 = kc<T>(c, KC_B10), b01 = kc<T>(c, KC_B01), b11 = kc<T>(c, KC_B11);
        const T rr_ = kc<T>(c, KC_R), inv_crho = kc<T>(c, KC_INV_CRHO), inv_aw = kc<T>(c, KC_INV_AW);
        const T P1 = kc<T>(c, KC_P1), P2 = kc<T>(c, KC_P2), psi1 = kc<T>(c, KC_PSI1), psi2 = kc<T>(c, KC_PSI2);
        for_tile_vectors<T>(g, it, [&](long long d, int cnt, int, int) {
            const Pack<T> f1 = ldv_n(P.f[RECON_F_F1], d, cnt), f2 = ldv_n(P.f[RECON_F_F2], d, cnt);
            const Pack<T> dr = ldv_n(P.f[RECON_F_DIV_RHO], d, cnt), dz = ldv_n(P.f[RECON_F_DIV_Z], d, cnt);
            Pack<T> orr, oa2, orz;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                // eq. mac_E1/E2 from the new fractions, then eq. rho_e and
                // eq. Z_m (normalised); the two nearly cancelling products of
                // a and b are formed with an exact split of one of them
                const T m1 = b00 * f1.v[e] + b10 * f2.v[e];
                const T m2 = b01 * f1.v[e] + b11 * f2.v[e];
                const T rho_cf = (m1 * rr_ - m2) * inv_crho;
                const T a = diff_of_products(m1, P2, m2, P1) * inv_aw;
                const T b = diff_of_products(m2, psi1, m1, psi2) * inv_aw;
                orr.v[e] = rho_cf + dr.v[e];
                oa2.v[e] = a * a;
                orz.v[e] = a * b + dz.v[e];
            }
            stv_n(P.f[RECON_F_RHS_RHO], d, orr, cnt);
            stv_n(P.f[RECON_F_A2], d, oa2, cnt);
            stv_n(P.f[RECON_F_RHS_Z], d, orz, cnt);
        });
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// PCG for [diag(a^2) + beta~ L] z = rhs
// --------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T lap5(const T (*sm)[TileDim<T>::SW], int ry, int cx) {
    const T c = sm[ry][cx];
    return (T(4) * c - sm[ry][cx - 1] - sm[ry][cx + 1]) - (sm[ry - 1][cx] + sm[ry + 1][cx]);
}

// --------------------------------------------------------------------------
// Multigrid preconditioner of the Z^m PCG
// --------------------------------------------------------------------------
// On slices whose sides halve down to a small grid, the PCG takes
// y = B r with B one V(1,1)-cycle for M = diag(a^2) + beta~ L: a damped
// Jacobi step (weight kMgOmega) before and after the coarse correction;
// coarse grids of half the sides, the residual and a^2 restricted as 2x2
// means, corrections prolonged piecewise constant, and beta~ / 4 per level
// (the Laplacian on a grid of twice the spacing).  The restriction is 1/4 of
// the transpose of the prolongation and both smoothing steps are the same
// Jacobi step, so B is symmetric positive definite, as PCG needs.  Levels of
// more than kMgBlockPx pixels run as tile kernels over all slices; the rest
// of the cycle of a slice runs inside one thread block (kMgBlockSweeps Jacobi
// steps before and after the correction there), with an exact solve
// on the coarsest grid (at most kMgCoarsePx pixels) by the inverse of its
// operator, formed once per Z^m solve.
// The fine-level passes of one PCG step:
//   k_mg_fwd   z += alpha p, r' = r - alpha q (into the other r buffer), r'.r'
//              and the convergence test; pre-smoothing x1 = w r' / (a^2 + 4 beta~)
//              and the restricted residual of level 1
//   k_mg_down  the same restriction on each tile level below (no update)
//   k_mg_block the levels of a slice that fit one block, and the coarsest solve
//   k_mg_up    coarse correction and post-smoothing on each tile level
//   k_mg_y     the same on the fine level: y = B r', r'.y -> beta_cg
//   k_mg_pq    p = y + beta_cg p_old, q = M p, p.q -> alpha

constexpr int kMgBlockPx = 4096;       // levels of at most this many pixels run inside one block
constexpr int kMgCoarsePx = 64;        // the coarsest grid has at most this many pixels
constexpr int kMgMaxBlockLevels = 8;
constexpr int kMgBlockSweeps = 2;      // Jacobi sweeps before and after the correction on the block's levels
constexpr int kMgBlockThreads = 256;
// k_mg_block: its passes stride over a level by the block size and hold no
// per-thread state across pixels, so the result does not depend on it; 512
// threads hide the shared-memory latency of a pass better, and two blocks
// still fit an SM (registers and the 64^2 levels' shared memory), so one
// block per slice runs in one wave for up to twice the SM count.
constexpr int kMgBlockRunThreads = 512;

// x / y for the Jacobi weights of the cycle: any fixed positive diagonal
// keeps the cycle symmetric, so FP32 kernels use the fast reciprocal.
__device__ __forceinline__ float mg_div(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double mg_div(double x, double y) { return x / y; }

// i mod n for i in [-n, 2n)
__device__ __forceinline__ int wrap_near(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// i mod n (non-negative) for any i: one compare and add in the common case
__device__ __forceinline__ int wrap_any(int i, int n) { return (i >= -n && i < 2 * n) ? wrap_near(i, n) : wrap(i, n); }

template <typename T>
__device__ __forceinline__ T mg_omega() {
    return T(0.8);
}

// beta~ / 4^lvl
template <typename T>
__device__ __forceinline__ T mg_bt(const SliceState& s, int lvl) {
    T b = Sc<T>::beta_t(s);
    for (int i = 0; i < lvl; ++i) b *= T(0.25);
    return b;
}

// fn(row, col) for every element of a shared-memory tile and its halo
template <typename T, typename F>
__device__ __forceinline__ void for_halo_tile(F fn) {
    constexpr int W = kTileW + 2, H = TileDim<T>::TH + 2, OFF = TileDim<T>::OFF;
    for (int q = threadIdx.x; q < W * H; q += blockDim.x) {
        const int ly = q / W, lx = q - ly * W;
        fn(ly, OFF - 1 + lx);
    }
}

// Grid of one slice at one level, read once per item by every thread.
struct TileGeo {
    long long off;
    int nx, ny, pitch, lvl;
};
__device__ __forceinline__ TileGeo tile_geo(const SliceGeom* G, int s) {
    const SliceGeom* g = G + s;
    return TileGeo{__ldg(&g->off), __ldg(&g->nx), __ldg(&g->ny), __ldg(&g->pitch), __ldg(&g->lvl)};
}

// A VN-vector of shared memory at a 16-byte aligned address.
template <typename T>
__device__ __forceinline__ Pack<T> lds_pack(const T* p) {
    return *reinterpret_cast<const Pack<T>*>(p);
}
template <typename T>
__device__ __forceinline__ void sts_pack(T* p, const Pack<T>& v) {
    *reinterpret_cast<Pack<T>*>(p) = v;
}

// Over a tile and its halo in shared memory: fv(row, c0) for the interior
// columns as VN-vectors (c0 = OFF + k VN), fs(row, col) for the two halo
// columns.
template <typename T, typename FV, typename FS>
__device__ __forceinline__ void for_halo_vec(FV fv, FS fs) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, H = TileDim<T>::TH + 2, VR = kTileW / VN;
    for (int q = threadIdx.x; q < H * VR; q += blockDim.x) {
        const int ry = q / VR;
        fv(ry, OFF + (q - ry * VR) * VN);
    }
    for (int q = threadIdx.x; q < 2 * H; q += blockDim.x) fs(q >> 1, (q & 1) ? OFF + kTileW : OFF - 1);
}

// (a^2 x + bt L x) for the VN pixels of row ry from column c0 (x in sx with
// its halo), given a^2 there.
// The Z^m operator at one pixel in FP32, a c + bt ((4c - l - r) - (u + d)):
// the one rounding sequence of every FP32 kernel that forms it (k_cg_init and
// the strip and band kernels), so that they agree bit for bit.
__device__ __forceinline__ float m_op(float a, float c, float l, float r, float u, float d, float bt) {
    const float lap = __fsub_rn(__fsub_rn(__fsub_rn(__fmul_rn(4.f, c), l), r), __fadd_rn(u, d));
    return __fmaf_rn(a, c, __fmul_rn(bt, lap));
}

template <typename T>
__device__ __forceinline__ Pack<T> mx_pack(const T (*sx)[TileDim<T>::SW], int ry, int c0, const Pack<T>& a, T bt,
                                           Pack<T>& xc) {
    constexpr int VN = TileDim<T>::VN;
    xc = lds_pack<T>(&sx[ry][c0]);
    const Pack<T> xu = lds_pack<T>(&sx[ry - 1][c0]), xd = lds_pack<T>(&sx[ry + 1][c0]);
    const T xl = sx[ry][c0 - 1], xr = sx[ry][c0 + VN];
    Pack<T> o;
#pragma unroll
    for (int e = 0; e < VN; ++e) {
        const T l = e == 0 ? xl : xc.v[e - 1];
        const T r = e == VN - 1 ? xr : xc.v[e + 1];
        if constexpr (std::is_same<T, float>::value) {
            o.v[e] = m_op(a.v[e], xc.v[e], l, r, xu.v[e], xd.v[e], bt);
        } else {
            const T lap = (T(4) * xc.v[e] - l - r) - (xu.v[e] + xd.v[e]);
            o.v[e] = a.v[e] * xc.v[e] + bt * lap;
        }
    }
    return o;
}

// Pre-smoothing from zero on the tile and its halo: x = w f / (a^2 + 4 bt).
template <typename T>
__device__ __forceinline__ void mg_presmooth(const T (*sf)[TileDim<T>::SW], const T (*sa)[TileDim<T>::SW],
                                             T (*sx)[TileDim<T>::SW], T om, T b4) {
    constexpr int VN = TileDim<T>::VN;
    for_halo_vec<T>(
        [&](int ry, int c0) {
            const Pack<T> f = lds_pack<T>(&sf[ry][c0]), a = lds_pack<T>(&sa[ry][c0]);
            Pack<T> x;
#pragma unroll
            for (int e = 0; e < VN; ++e) x.v[e] = mg_div(om * f.v[e], a.v[e] + b4);
            sts_pack<T>(&sx[ry][c0], x);
        },
        [&](int ry, int c) { sx[ry][c] = mg_div(om * sf[ry][c], sa[ry][c] + b4); });
}

// Restricted residual of the tile at (tx0, ty0) of level g: out at level g1 =
// mean over each 2x2 block of f - (a^2 x + bt L x), with f, a^2, x on the tile
// and its halo in shared memory.
template <typename T>
__device__ __forceinline__ void mg_restrict_residual(const T (*sf)[TileDim<T>::SW], const T (*sa)[TileDim<T>::SW],
                                                     const T (*sx)[TileDim<T>::SW], const TileGeo& g,
                                                     const TileGeo& g1, int tx0, int ty0, T bt, T* out) {
    // one task: two fine rows x VN fine columns = VN / 2 coarse cells
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, CH = TileDim<T>::TH / 2, VR = kTileW / VN;
    for (int q = threadIdx.x; q < CH * VR; q += blockDim.x) {
        const int cy = q / VR, k = q - cy * VR;
        const int x0 = tx0 + k * VN;
        if (x0 >= g.nx || ty0 + 2 * cy >= g.ny) continue;
        const int c0 = OFF + k * VN;
        T sum[VN / 2];
#pragma unroll
        for (int i = 0; i < VN / 2; ++i) sum[i] = T(0);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int ry = 1 + 2 * cy + dy;
            const Pack<T> a = lds_pack<T>(&sa[ry][c0]), f = lds_pack<T>(&sf[ry][c0]);
            Pack<T> xc;
            const Pack<T> m = mx_pack<T>(sx, ry, c0, a, bt, xc);
#pragma unroll
            for (int e = 0; e < VN; ++e) sum[e >> 1] += f.v[e] - m.v[e];
        }
        T* o = out + g1.off + (long long)(ty0 / 2 + cy) * g1.pitch + x0 / 2;
#pragma unroll
        for (int i = 0; i < VN / 2; ++i)
            if (x0 + 2 * i < g.nx) o[i] = T(0.25) * sum[i];
    }
}

// a^2 of level g1 = 2x2 means of level g (tiles of level g)
template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_mg_restrict(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                                 const SliceState* S, const T* a, T* a1,
                                                                 unsigned long long* acct) {
    constexpr int CW = kTileW / 2, CH = TileDim<T>::TH / 2;
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        if (!__ldg(&S[it.slice].active)) continue;
        const SliceGeom g = G[it.slice], g1 = G1[it.slice];
        account(acct, KF_MG_SETUP, tile_px<T>(g, it) * 5 * (long long)sizeof(T) / 4);
        for (int q = threadIdx.x; q < CW * CH; q += blockDim.x) {
            const int cy = q / CW, cx = q - cy * CW;
            const int x = it.a + 2 * cx, y = it.b + 2 * cy;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            a1[g1.off + (long long)(y / 2) * g1.pitch + x / 2] =
                T(0.25) * ((a[d] + a[d + 1]) + (a[d + g.pitch] + a[d + g.pitch + 1]));
        }
    }
}

// Level geometries 0 .. n of the a^2 restriction (device arrays, one entry per slice).
constexpr int kMgRestrictFused = 5;   // most levels one fine tile forms in k_mg_restrict_all (64 x 32 -> 2 x 1)
struct MgLevelGeoms {
    const SliceGeom* g[kMgRestrictFused + 1];
};

// a^2 of levels 1 .. nlev from the fine a^2 in one pass over the fine tiles:
// a tile's 2x2 means of level l are formed from its level-l cells in shared
// memory (the tile's own cells: 2x2 means stay within a tile whose sides are
// multiples of 2^nlev), each written to its level.  Every value is the sum
// k_mg_restrict forms from the same four values, so the levels equal those of
// one k_mg_restrict launch per level, bit for bit.  A slice stops at its own
// depth (the next level's width is 0).
template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_mg_restrict_all(ItemList L, MgLevelGeoms LG, int nlev,
                                                                     const SliceState* S, const T* a, T* pa,
                                                                     unsigned long long* acct) {
    constexpr int TH = TileDim<T>::TH;
    __shared__ T sm[2][TH / 2][kTileW / 2];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        if (!__ldg(&S[it.slice].active)) continue;
        const SliceGeom g = LG.g[0][it.slice], g1 = LG.g[1][it.slice];
        account(acct, KF_MG_SETUP, tile_px<T>(g, it) * 5 * (long long)sizeof(T) / 4);
        int cw = kTileW / 2, ch = TH / 2;
        for (int q = threadIdx.x; q < cw * ch; q += blockDim.x) {
            const int cy = q / cw, cx = q - cy * cw;
            const int x = it.a + 2 * cx, y = it.b + 2 * cy;
            T v = T(0);
            if (x < g.nx && y < g.ny) {
                const long long d = g.off + (long long)y * g.pitch + x;
                v = T(0.25) * ((a[d] + a[d + 1]) + (a[d + g.pitch] + a[d + g.pitch + 1]));
                pa[g1.off + (long long)(y / 2) * g1.pitch + x / 2] = v;
            }
            sm[0][cy][cx] = v;
        }
        __syncthreads();
        int buf = 0;
        for (int l = 1; l < nlev && (ch >> 1) > 0; ++l) {
            const SliceGeom gl = LG.g[l][it.slice], gn = LG.g[l + 1][it.slice];
            if (gn.nx == 0) break;   // the slice has no level l + 1 (the same for the whole block)
            const int x0 = it.a >> l, y0 = it.b >> l;   // the tile's origin on level l
            {
                const int w = gl.nx - x0 < cw ? gl.nx - x0 : cw, h = gl.ny - y0 < ch ? gl.ny - y0 : ch;
                const long long px = (long long)(w > 0 ? w : 0) * (h > 0 ? h : 0);
                account(acct, KF_MG_SETUP, px * 5 * (long long)sizeof(T) / 4);
            }
            cw >>= 1;
            ch >>= 1;
            for (int q = threadIdx.x; q < cw * ch; q += blockDim.x) {
                const int cy = q / cw, cx = q - cy * cw;
                const int x = x0 + 2 * cx, y = y0 + 2 * cy;
                T v = T(0);
                if (x < gl.nx && y < gl.ny) {
                    v = T(0.25) * ((sm[buf][2 * cy][2 * cx] + sm[buf][2 * cy][2 * cx + 1]) +
                                   (sm[buf][2 * cy + 1][2 * cx] + sm[buf][2 * cy + 1][2 * cx + 1]));
                    pa[gn.off + (long long)(y / 2) * gn.pitch + x / 2] = v;
                }
                sm[buf ^ 1][cy][cx] = v;
            }
            __syncthreads();
            buf ^= 1;
        }
    }
}

// Start the copies of NM maps of the tile at (tx0, ty0) with its one-pixel
// periodic halo into sm[m] (layout of load_tile).
template <typename T, int NM>
__device__ __forceinline__ void halo_async(T (*sm)[TileDim<T>::TH + 2][TileDim<T>::SW], const TileGeo& g, int tx0,
                                           int ty0, const T* const (&src)[NM], int nm = NM) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, TH = TileDim<T>::TH, VR = kTileW / VN;
    if (tx0 + kTileW <= g.nx) {
        for (int q = threadIdx.x; q < (TH + 2) * VR; q += blockDim.x) {
            const int ly = q / VR, lx = (q - ly * VR) * VN;
            const long long d = g.off + (long long)wrap_any(ty0 - 1 + ly, g.ny) * g.pitch + tx0 + lx;
#pragma unroll
            for (int m = 0; m < NM; ++m)
                if (m < nm) cp_async16(&sm[m][ly][OFF + lx], src[m] + d);
        }
        for (int q = threadIdx.x; q < 2 * (TH + 2); q += blockDim.x) {
            const int ly = q >> 1, side = q & 1;
            const int gx = side ? wrap_any(tx0 + kTileW, g.nx) : wrap_any(tx0 - 1, g.nx);
            const long long d = g.off + (long long)wrap_any(ty0 - 1 + ly, g.ny) * g.pitch + gx;
#pragma unroll
            for (int m = 0; m < NM; ++m)
                if (m < nm) cp_async_elem<sizeof(T)>(&sm[m][ly][side ? OFF + kTileW : OFF - 1], src[m] + d);
        }
    } else {
        for (int q = threadIdx.x; q < (TH + 2) * (kTileW + 2); q += blockDim.x) {
            const int ly = q / (kTileW + 2), lx = q - ly * (kTileW + 2);
            const long long d =
                g.off + (long long)wrap(ty0 - 1 + ly, g.ny) * g.pitch + wrap(tx0 - 1 + lx, g.nx);
#pragma unroll
            for (int m = 0; m < NM; ++m)
                if (m < nm) cp_async_elem<sizeof(T)>(&sm[m][ly][OFF - 1 + lx], src[m] + d);
        }
    }
}

// Start the copies of NM maps of the tile interior into si[m][ly][lx].
template <typename T, int NM>
__device__ __forceinline__ void inner_async(T (*si)[TileDim<T>::TH][kTileW], const TileGeo& g, int tx0, int ty0,
                                            const T* const (&src)[NM]) {
    constexpr int VN = TileDim<T>::VN, TH = TileDim<T>::TH, VR = kTileW / VN;
    for (int q = threadIdx.x; q < TH * VR; q += blockDim.x) {
        const int ly = q / VR, lx = (q - ly * VR) * VN;
        const int y = ty0 + ly, x0 = tx0 + lx;
        if (y >= g.ny || x0 >= g.nx) continue;
        const long long d = g.off + (long long)y * g.pitch + x0;
        if (x0 + VN <= g.nx) {
#pragma unroll
            for (int m = 0; m < NM; ++m) cp_async16(&si[m][ly][lx], src[m] + d);
        } else {
            for (int e = 0; e < g.nx - x0; ++e)
#pragma unroll
                for (int m = 0; m < NM; ++m) cp_async_elem<sizeof(T)>(&si[m][ly][lx + e], src[m] + d + e);
        }
    }
}

// Start the copies of the coarse cells under a tile of the finer level and
// its halo (periodic on the coarse grid g1) into ec.
template <typename T>
__device__ __forceinline__ void coarse_async(T (*ec)[kTileW / 2 + 2], const TileGeo& g1, int tx0, int ty0,
                                             const T* E1) {
    constexpr int CH = TileDim<T>::TH / 2 + 2, CW = kTileW / 2 + 2;
    const int X0 = tx0 / 2 - 1, Y0 = ty0 / 2 - 1;
    for (int q = threadIdx.x; q < CH * CW; q += blockDim.x) {
        const int cy = q / CW, cx = q - cy * CW;
        cp_async_elem<sizeof(T)>(
            &ec[cy][cx], E1 + g1.off + (long long)wrap_any(Y0 + cy, g1.ny) * g1.pitch + wrap_any(X0 + cx, g1.nx));
    }
}

// An item of a pipelined stencil kernel: the tile, its slice's grid(s) and
// whether it runs (slice active, PCG not converged).
struct PipeItem {
    Item it;
    TileGeo g, g1;
    int first;   // PCG step count is 0
    bool ok;
};

// Persistent loop over the items of L in which the copies of the next item
// run while the current one is computed (two buffers).  make(item) fills a
// PipeItem, issue(p, buf) starts the copies of p, compute(p, buf, index)
// runs with the copies of p complete.  Item descriptors are read two items
// ahead.  Every thread of the block takes the same path.
template <typename Buf, typename FM, typename FI, typename FC>
__device__ __forceinline__ void pipeline_items(const ItemList& L, Buf* buf, FM make, FI issue, FC compute) {
    const int step = gridDim.x, n = L.n_items;
    int w = blockIdx.x;
    if (w >= n) return;
    PipeItem cur = make(L.items[w]);
    Item i1 = w + step < n ? L.items[w + step] : Item{};
    if (cur.ok) issue(cur, buf[0]);
    cp_async_commit();
    for (int k = 0; w < n; w += step, k ^= 1) {
        PipeItem nxt;
        nxt.ok = false;
        if (w + step < n) {
            nxt = make(i1);
            if (w + 2 * step < n) i1 = L.items[w + 2 * step];
            if (nxt.ok) issue(nxt, buf[k ^ 1]);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (cur.ok) compute(cur, buf[k], w);
        __syncthreads();
        cur = nxt;
    }
    cp_async_wait<0>();
}

// ---- start of the Z^m PCG: r = rhs - M z, with mean(a^2), ||rhs||^2, r.r ----

template <typename T>
struct CgInitBuf {
    T h[1][TileDim<T>::TH + 2][TileDim<T>::SW];   // z with halo
    T in[2][TileDim<T>::TH][kTileW];              // a^2, rhs
};

template <typename T>
__global__ void __launch_bounds__(kStencilThreads, 4) k_cg_init(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                             SliceState* S, Ptrs<T> P, int* pending) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, TH = TileDim<T>::TH, VR = kTileW / VN;
    extern __shared__ __align__(16) unsigned char cg_dsm[];
    CgInitBuf<T>* buf = reinterpret_cast<CgInitBuf<T>*>(cg_dsm);
    __shared__ double red[3 * 32];
    const T* z = P.f[RECON_F_Z];
    const T* a2 = P.f[RECON_F_A2];
    const T* rz = P.f[RECON_F_RHS_Z];
    T* r = P.f[RECON_F_CG_R];
    auto make = [&](const Item& it) {
        PipeItem p;
        p.it = it;
        p.first = 0;
        p.ok = __ldg(&S[it.slice].active);
        if (p.ok) p.g = tile_geo(G, it.slice);
        return p;
    };
    auto issue = [&](const PipeItem& c, CgInitBuf<T>& b) {
        const T* hs[1] = {z};
        halo_async<T, 1>(b.h, c.g, c.it.a, c.it.b, hs);
        const T* is[2] = {a2, rz};
        inner_async<T, 2>(b.in, c.g, c.it.a, c.it.b, is);
    };
    auto compute = [&](const PipeItem& c, CgInitBuf<T>& b, int w) {
        const TileGeo& g = c.g;
        account(P.acct, KF_CG_INIT,
                (long long)min(TH, g.ny - c.it.b) * min(kTileW, g.nx - c.it.a) * 4 * (long long)sizeof(T));
        const T bt = Sc<T>::beta_t(S[c.it.slice]);
        T accT = T(0), acc_a2 = T(0), acc_b = T(0);
        for (int q = threadIdx.x; q < TH * VR; q += blockDim.x) {
            const int ly = q / VR, lx0 = (q - ly * VR) * VN;
            const int y = c.it.b + ly, x0 = c.it.a + lx0;
            if (y >= g.ny || x0 >= g.nx) continue;
            const int cnt = g.nx - x0 < VN ? g.nx - x0 : VN;
            const Pack<T> av = lds_pack<T>(&b.in[0][ly][lx0]), bv = lds_pack<T>(&b.in[1][ly][lx0]);
            Pack<T> zc;
            const Pack<T> m = mx_pack<T>(b.h[0], ly + 1, OFF + lx0, av, bt, zc);
            Pack<T> rv;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                rv.v[e] = sub_rn(bv.v[e], m.v[e]);
                if (e < cnt) {
                    accT = fma(rv.v[e], rv.v[e], accT);
                    acc_a2 += av.v[e];
                    acc_b = fma(bv.v[e], bv.v[e], acc_b);
                }
            }
            stv_n(r, g.off + (long long)y * g.pitch + x0, rv, cnt);
        }
        const T part[3] = {accT, acc_a2, acc_b};
        double acc[3];
        block_sum_t<T, 3>(part, acc, red);
        double tot[3];
        if (item_reduce<3>(L, w, c.it.slice, acc, tot, red)) {
            SliceState& so = S[c.it.slice];
            const double tol2 = C[c.it.slice].cg_tol * C[c.it.slice].cg_tol;
            // mean(a^2) sets the preconditioner's diagonal, ||rhs||^2 the
            // stopping test (of the a^2 and rhs this solve reads)
            set_abar2(so, tot[1] / ((double)g.nx * (double)g.ny));
            so.bb = tot[2];
            so.rr = tot[0];
            so.rr0 = tot[0];
            so.cg_it = 0;
            so.ry = 0.0;
            set_betacg(so, 0.0);
            so.cg_done = (so.bb == 0.0 || !(tot[0] > tol2 * so.bb)) ? 1 : 0;
            if (!so.cg_done) atomicAdd(pending, 1);
        }
    };
    pipeline_items(L, buf, make, issue, compute);
}

// x on the tile and its halo (sx) = w f / (a^2 + 4 bt) + e1 (the coarse
// correction of level g1, constant on 2x2 blocks, from ec); then for each
// pixel of the tile x + w (f - (a^2 x + bt L x)) / (a^2 + 4 bt), passed to
// out(d, cnt, ly, lx0, value pack).  sf, sa: f and a^2 on the tile and halo.
template <typename T, typename FO>
__device__ __forceinline__ void mg_correct_smooth(const T (*sf)[TileDim<T>::SW], const T (*sa)[TileDim<T>::SW],
                                                  T (*sx)[TileDim<T>::SW], const T (*ec)[kTileW / 2 + 2],
                                                  const TileGeo& g, const Item& it, T bt, FO out) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, TH = TileDim<T>::TH, VR = kTileW / VN;
    const T b4 = T(4) * bt, om = mg_omega<T>();
    // tile row ry is pixel row it.b - 1 + ry: coarse row (ry + 1) >> 1 of ec;
    // column c is coarse column (c - OFF + 2) >> 1
    for_halo_vec<T>(
        [&](int ry, int c0) {
            const Pack<T> f = lds_pack<T>(&sf[ry][c0]), a = lds_pack<T>(&sa[ry][c0]);
            const T* e = ec[(ry + 1) >> 1];
            Pack<T> x;
#pragma unroll
            for (int i = 0; i < VN; ++i) x.v[i] = mg_div(om * f.v[i], a.v[i] + b4) + e[(c0 + i - OFF + 2) >> 1];
            sts_pack<T>(&sx[ry][c0], x);
        },
        [&](int ry, int c) {
            sx[ry][c] = mg_div(om * sf[ry][c], sa[ry][c] + b4) + ec[(ry + 1) >> 1][(c - OFF + 2) >> 1];
        });
    __syncthreads();
    for (int q = threadIdx.x; q < TH * VR; q += blockDim.x) {
        const int ly = q / VR, lx0 = (q - ly * VR) * VN;
        const int y = it.b + ly, x0 = it.a + lx0;
        if (y >= g.ny || x0 >= g.nx) continue;
        const int cnt = g.nx - x0 < VN ? g.nx - x0 : VN;
        const int ry = ly + 1, c0 = OFF + lx0;
        const Pack<T> a = lds_pack<T>(&sa[ry][c0]), f = lds_pack<T>(&sf[ry][c0]);
        Pack<T> xc;
        const Pack<T> m = mx_pack<T>(sx, ry, c0, a, bt, xc);
        Pack<T> o;
#pragma unroll
        for (int e = 0; e < VN; ++e) o.v[e] = xc.v[e] + mg_div(om * (f.v[e] - m.v[e]), a.v[e] + b4);
        out(g.off + (long long)y * g.pitch + x0, cnt, ly, lx0, o);
    }
}

template <typename T>
struct MgBufFwd {   // r, a^2, q with halo
    T h[3][TileDim<T>::TH + 2][TileDim<T>::SW];
};
template <typename T>
struct MgBufHalo2 {   // f (or r), a^2 with halo; the coarse correction under the tile
    T h[2][TileDim<T>::TH + 2][TileDim<T>::SW];
    T ec[TileDim<T>::TH / 2 + 2][kTileW / 2 + 2];
};
template <typename T>
struct MgBufPq {   // y, p_old with halo; a^2 interior
    T h[2][TileDim<T>::TH + 2][TileDim<T>::SW];
    T in[1][TileDim<T>::TH][kTileW];
};

// PipeItem of a multigrid kernel: slice active and its PCG not converged.
__device__ __forceinline__ PipeItem mg_item(const Item& it, const SliceGeom* G, const SliceGeom* G1,
                                            const SliceState* S) {
    PipeItem p;
    p.it = it;
    const SliceState* sp = S + it.slice;
    p.ok = __ldg(&sp->active) && !__ldg(&sp->cg_done);
    p.first = __ldg(&sp->cg_it) == 0;
    if (p.ok) {
        p.g = tile_geo(G, it.slice);
        if (G1) p.g1 = tile_geo(G1, it.slice);
    }
    return p;
}

// Fine level, start of a PCG step (UPD: after the update with alpha).  r is
// read from rin and, updated, written to rout: other tiles read the old r on
// their halo in the same launch.
template <typename T, bool UPD>
__global__ void __launch_bounds__(kStencilThreads, 3) k_mg_fwd(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                             const SliceConst* C, SliceState* S, Ptrs<T> P, int par,
                                                             const T* rin, T* rout, T* F1, int* pending) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, TH = TileDim<T>::TH;
    extern __shared__ __align__(16) unsigned char mg_dsm[];
    MgBufFwd<T>* buf = reinterpret_cast<MgBufFwd<T>*>(mg_dsm);
    __shared__ double red[32];
    T* z = P.f[RECON_F_Z];
    const T* p = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    const T* q = P.f[RECON_F_CG_Q];
    const T* a2 = P.f[RECON_F_A2];
    auto make = [&](const Item& it) { return mg_item(it, G, G1, S); };
    auto issue = [&](const PipeItem& c, MgBufFwd<T>& b) {
        const T* hs[3] = {rin, a2, q};
        halo_async<T, 3>(b.h, c.g, c.it.a, c.it.b, hs, UPD ? 3 : 2);
    };
    struct In {
        Pack<T> z, p;
    };
    auto load = [&](long long d, int cnt) { return In{ldv_n(z, d, cnt), ldv_n(p, d, cnt)}; };
    auto compute = [&](const PipeItem& c, MgBufFwd<T>& b, int w) {
        const TileGeo& g = c.g;
        const SliceState* sp = S + c.it.slice;
        account(P.acct, KF_MG_FWD,
                (long long)min(TH, g.ny - c.it.b) * min(kTileW, g.nx - c.it.a) * (UPD ? 29 : 9) * (long long)sizeof(T) /
                    4);
        const T bt = Sc<T>::beta_t(*sp), b4 = Sc<T>::b4(*sp), om = mg_omega<T>();
        T acc = T(0);
        if (UPD) {
            // z and p are pointwise: loaded into registers, in flight during the r update
            const SliceGeom gs{g.nx, g.ny, g.pitch, 0, 0, g.off};
            In v[TileVec<T>::R];
            tile_vec_load<T>(gs, c.it, load, v);
            const T al = Sc<T>::alpha(*sp);
            for_halo_vec<T>(
                [&](int ry, int c0) {
                    Pack<T> r = lds_pack<T>(&b.h[0][ry][c0]);
                    const Pack<T> qv = lds_pack<T>(&b.h[2][ry][c0]);
#pragma unroll
                    for (int e = 0; e < VN; ++e) r.v[e] = fma(-al, qv.v[e], r.v[e]);
                    sts_pack<T>(&b.h[0][ry][c0], r);
                },
                [&](int ry, int col) { b.h[0][ry][col] = fma(-al, b.h[2][ry][col], b.h[0][ry][col]); });
            __syncthreads();
            tile_vec_use<T>(
                gs, c.it,
                [&](long long d, int cnt, int ly, int lx0, const In& x) {
                    Pack<T> zn, rn;
#pragma unroll
                    for (int e = 0; e < VN; ++e) {
                        zn.v[e] = fma(al, x.p.v[e], x.z.v[e]);
                        rn.v[e] = b.h[0][ly + 1][OFF + lx0 + e];
                        if (e < cnt) acc = fma(rn.v[e], rn.v[e], acc);
                    }
                    stv_n(z, d, zn, cnt);
                    stv_n(rout, d, rn, cnt);
                },
                v);
        }
        // pre-smoothing from zero, on the tile and its halo (in place of q)
        mg_presmooth<T>(b.h[0], b.h[1], b.h[2], om, b4);
        __syncthreads();
        mg_restrict_residual<T>(b.h[0], b.h[1], b.h[2], g, c.g1, c.it.a, c.it.b, bt, F1);
        if (UPD) {
            const T part[1] = {acc};
            double a[1];
            block_sum_t<T, 1>(part, a, red);
            double tot[1];
            if (item_reduce<1>(L, w, c.it.slice, a, tot, red)) {
                SliceState& so = S[c.it.slice];
                const SliceConst& cs = C[c.it.slice];
                so.rr = tot[0];
                so.cg_it += 1;
                const bool conv = !(tot[0] > cs.cg_tol * cs.cg_tol * so.bb);
                if (conv || so.cg_it >= cs.cg_max) {
                    so.cg_done = 1;
                    atomicSub(pending, 1);
                    atomicMax(pending + 1, so.cg_it);
                }
            }
        }
    };
    pipeline_items(L, buf, make, issue, compute);
}

// Tile level g (level >= 1): pre-smoothing from zero and the restricted
// residual into level g1.
template <typename T>
__global__ void __launch_bounds__(kStencilThreads, 4) k_mg_down(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                              const SliceState* S, const T* F, const T* A, T* F1,
                                                              unsigned long long* acct) {
    constexpr int TH = TileDim<T>::TH;
    extern __shared__ __align__(16) unsigned char mg_dsm[];
    MgBufHalo2<T>* buf = reinterpret_cast<MgBufHalo2<T>*>(mg_dsm);
    __shared__ __align__(16) T sx[TH + 2][TileDim<T>::SW];
    auto make = [&](const Item& it) { return mg_item(it, G, G1, S); };
    auto issue = [&](const PipeItem& c, MgBufHalo2<T>& b) {
        const T* hs[2] = {F, A};
        halo_async<T, 2>(b.h, c.g, c.it.a, c.it.b, hs);
    };
    auto compute = [&](const PipeItem& c, MgBufHalo2<T>& b, int) {
        const TileGeo& g = c.g;
        account(acct, KF_MG_LEVELS,
                (long long)min(TH, g.ny - c.it.b) * min(kTileW, g.nx - c.it.a) * 9 * (long long)sizeof(T) / 4);
        const T bt = mg_bt<T>(S[c.it.slice], g.lvl), b4 = T(4) * bt, om = mg_omega<T>();
        mg_presmooth<T>(b.h[0], b.h[1], sx, om, b4);
        __syncthreads();
        mg_restrict_residual<T>(b.h[0], b.h[1], sx, g, c.g1, c.it.a, c.it.b, bt, F1);
    };
    pipeline_items(L, buf, make, issue, compute);
}

// Tile level g (level >= 1): e = coarse correction and post-smoothing.
template <typename T>
__global__ void __launch_bounds__(kStencilThreads, 4) k_mg_up(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                            const SliceState* S, const T* F, const T* A,
                                                            const T* E1, T* E, unsigned long long* acct) {
    constexpr int TH = TileDim<T>::TH;
    extern __shared__ __align__(16) unsigned char mg_dsm[];
    MgBufHalo2<T>* buf = reinterpret_cast<MgBufHalo2<T>*>(mg_dsm);
    __shared__ __align__(16) T sx[TH + 2][TileDim<T>::SW];
    auto make = [&](const Item& it) { return mg_item(it, G, G1, S); };
    auto issue = [&](const PipeItem& c, MgBufHalo2<T>& b) {
        const T* hs[2] = {F, A};
        halo_async<T, 2>(b.h, c.g, c.it.a, c.it.b, hs);
        coarse_async<T>(b.ec, c.g1, c.it.a, c.it.b, E1);
    };
    auto compute = [&](const PipeItem& c, MgBufHalo2<T>& b, int) {
        const TileGeo& g = c.g;
        account(acct, KF_MG_LEVELS,
                (long long)min(TH, g.ny - c.it.b) * min(kTileW, g.nx - c.it.a) * 13 * (long long)sizeof(T) / 4);
        mg_correct_smooth<T>(b.h[0], b.h[1], sx, b.ec, g, c.it, mg_bt<T>(S[c.it.slice], g.lvl),
                             [&](long long d, int cnt, int, int, const Pack<T>& o) { stv_n(E, d, o, cnt); });
    };
    pipeline_items(L, buf, make, issue, compute);
}

// Fine level: y = B r (correction from level 1 and post-smoothing), r.y ->
// beta_cg.
template <typename T>
__global__ void __launch_bounds__(kStencilThreads, 4) k_mg_y(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                           SliceState* S, Ptrs<T> P, const T* r, const T* E1) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, TH = TileDim<T>::TH;
    extern __shared__ __align__(16) unsigned char mg_dsm[];
    MgBufHalo2<T>* buf = reinterpret_cast<MgBufHalo2<T>*>(mg_dsm);
    __shared__ __align__(16) T sx[TH + 2][TileDim<T>::SW];
    __shared__ double red[32];
    const T* a2 = P.f[RECON_F_A2];
    T* y = P.f[RECON_F_CG_Y];
    auto make = [&](const Item& it) { return mg_item(it, G, G1, S); };
    auto issue = [&](const PipeItem& c, MgBufHalo2<T>& b) {
        const T* hs[2] = {r, a2};
        halo_async<T, 2>(b.h, c.g, c.it.a, c.it.b, hs);
        coarse_async<T>(b.ec, c.g1, c.it.a, c.it.b, E1);
    };
    auto compute = [&](const PipeItem& c, MgBufHalo2<T>& b, int w) {
        const TileGeo& g = c.g;
        account(P.acct, KF_MG_Y,
                (long long)min(TH, g.ny - c.it.b) * min(kTileW, g.nx - c.it.a) * 13 * (long long)sizeof(T) / 4);
        T acc = T(0);
        mg_correct_smooth<T>(b.h[0], b.h[1], sx, b.ec, g, c.it, Sc<T>::beta_t(S[c.it.slice]),
                             [&](long long d, int cnt, int ly, int lx0, const Pack<T>& o) {
#pragma unroll
                                 for (int e = 0; e < VN; ++e)
                                     if (e < cnt) acc = fma(b.h[0][ly + 1][OFF + lx0 + e], o.v[e], acc);
                                 stv_n(y, d, o, cnt);
                             });
        const T part[1] = {acc};
        double a[1];
        block_sum_t<T, 1>(part, a, red);
        double tot[1];
        if (item_reduce<1>(L, w, c.it.slice, a, tot, red)) {
            SliceState& so = S[c.it.slice];
            set_betacg(so, (so.cg_it == 0) ? 0.0 : tot[0] / so.ry);
            so.ry = tot[0];
        }
    };
    pipeline_items(L, buf, make, issue, compute);
}

// Fine level: p = y + beta_cg p_old (p = y on the first step), q = M p, p.q
// -> alpha.
template <typename T>
__global__ void __launch_bounds__(kStencilThreads, 4) k_mg_pq(ItemList L, const SliceGeom* G, SliceState* S,
                                                            Ptrs<T> P, int par) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, TH = TileDim<T>::TH, VR = kTileW / VN;
    extern __shared__ __align__(16) unsigned char mg_dsm[];
    MgBufPq<T>* buf = reinterpret_cast<MgBufPq<T>*>(mg_dsm);
    __shared__ double red[32];
    const T* y = P.f[RECON_F_CG_Y];
    const T* pold = P.f[par ? RECON_F_CG_P1 : RECON_F_CG_P0];
    T* pnew = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    const T* a2 = P.f[RECON_F_A2];
    T* qo = P.f[RECON_F_CG_Q];
    auto make = [&](const Item& it) { return mg_item(it, G, nullptr, S); };
    auto issue = [&](const PipeItem& c, MgBufPq<T>& b) {
        const T* hs[2] = {y, pold};
        halo_async<T, 2>(b.h, c.g, c.it.a, c.it.b, hs, c.first ? 1 : 2);   // no p_old on the first step
        const T* is[1] = {a2};
        inner_async<T, 1>(b.in, c.g, c.it.a, c.it.b, is);
    };
    auto compute = [&](const PipeItem& c, MgBufPq<T>& b, int w) {
        const TileGeo& g = c.g;
        const SliceState* sp = S + c.it.slice;
        account(P.acct, KF_MG_PQ,
                (long long)min(TH, g.ny - c.it.b) * min(kTileW, g.nx - c.it.a) * (c.first ? 4 : 5) *
                    (long long)sizeof(T));
        if (!c.first) {
            const T bc = Sc<T>::betacg(*sp);
            for_halo_vec<T>(
                [&](int ry, int c0) {
                    Pack<T> pv = lds_pack<T>(&b.h[0][ry][c0]);
                    const Pack<T> po = lds_pack<T>(&b.h[1][ry][c0]);
#pragma unroll
                    for (int e = 0; e < VN; ++e) pv.v[e] = fma(bc, po.v[e], pv.v[e]);
                    sts_pack<T>(&b.h[0][ry][c0], pv);
                },
                [&](int ry, int col) { b.h[0][ry][col] = fma(bc, b.h[1][ry][col], b.h[0][ry][col]); });
            __syncthreads();
        }
        const T bt = Sc<T>::beta_t(*sp);
        T acc = T(0);
        for (int qq = threadIdx.x; qq < TH * VR; qq += blockDim.x) {
            const int ly = qq / VR, lx0 = (qq - ly * VR) * VN;
            const int yy = c.it.b + ly, x0 = c.it.a + lx0;
            if (yy >= g.ny || x0 >= g.nx) continue;
            const int cnt = g.nx - x0 < VN ? g.nx - x0 : VN;
            Pack<T> pv;
            const Pack<T> qv = mx_pack<T>(b.h[0], ly + 1, OFF + lx0, lds_pack<T>(&b.in[0][ly][lx0]), bt, pv);
#pragma unroll
            for (int e = 0; e < VN; ++e)
                if (e < cnt) acc = fma(pv.v[e], qv.v[e], acc);
            const long long d = g.off + (long long)yy * g.pitch + x0;
            stv_n(pnew, d, pv, cnt);
            stv_n(qo, d, qv, cnt);
        }
        const T part[1] = {acc};
        double a[1];
        block_sum_t<T, 1>(part, a, red);
        double tot[1];
        if (item_reduce<1>(L, w, c.it.slice, a, tot, red)) {
            SliceState& so = S[c.it.slice];
            so.pq = tot[0];
            set_alpha(so, tot[0] > 0.0 ? so.ry / tot[0] : 0.0);
        }
    };
    pipeline_items(L, buf, make, issue, compute);
}

}  // namespace recon
#include "mg_strip.cuh"
#include "mg_band.cuh"
#include "thr_band.cuh"
namespace recon {

// Sides of the in-block levels of a block level of bx x by pixels: halve while
// both sides are even and the grid has more than kMgCoarsePx pixels.
__host__ __device__ inline int mg_block_levels(int bx, int by, int* nx, int* ny) {
    int j = 0;
    nx[0] = bx;
    ny[0] = by;
    while (nx[j] * ny[j] > kMgCoarsePx && nx[j] % 2 == 0 && ny[j] % 2 == 0 && j + 1 < kMgMaxBlockLevels) {
        nx[j + 1] = nx[j] / 2;
        ny[j + 1] = ny[j] / 2;
        ++j;
    }
    return j + 1;
}

// Inverse of the coarsest operator diag(a^2) + bt L of each multigrid slice
// (once per Z^m solve; grid: one block per slice): a^2 restricted through
// the slice's block levels as in k_mg_block, the dense n x n operator
// (n <= kMgCoarsePx, periodic neighbours accumulate) inverted in the
// kernel's precision by Gauss-Jordan elimination without pivoting (the
// matrix is symmetric positive definite; its condition number stays below
// about 1e4, so FP32 keeps the inverse to about 1e-3, ample for a
// preconditioner), symmetrised, stored n x n.  Thread t keeps row t / 4 of
// the matrix (padded to kMgCoarsePx with identity rows), columns
// kMgInvCols (t % 4) onward, in registers; a pivot step publishes column k
// and the scaled pivot row through shared memory (two barriers a step).
constexpr int kMgInvCols = kMgCoarsePx / 4;
static_assert(kMgBlockThreads == 4 * kMgCoarsePx, "one row of the coarsest operator per four threads");
constexpr int kMgCoarseInvSmem =
    (kMgCoarsePx * (kMgCoarsePx + 1) + 2 * kMgCoarsePx) * (int)sizeof(double);   // + the a^2 of the levels

template <typename T>
__global__ void __launch_bounds__(kMgBlockThreads) k_mg_coarse_inv(const SliceGeom* GB, const SliceState* S,
                                                                   const T* A, T* Qinv) {
    extern __shared__ __align__(16) unsigned char mgq_smem[];
    T(*M)[kMgCoarsePx + 1] = reinterpret_cast<T(*)[kMgCoarsePx + 1]>(mgq_smem);
    T* fac = reinterpret_cast<T*>(mgq_smem) + kMgCoarsePx * (kMgCoarsePx + 1);
    T* a = reinterpret_cast<T*>(mgq_smem + kMgCoarseInvSmem);   // every level (sum of sizes)
    const int s = blockIdx.x;
    const SliceGeom g = GB[s];
    if (g.nx == 0 || !__ldg(&S[s].active)) return;
    int nx[kMgMaxBlockLevels], ny[kMgMaxBlockLevels], base[kMgMaxBlockLevels];
    const int J = mg_block_levels(g.nx, g.ny, nx, ny);
    int tot = 0;
    for (int j = 0; j < J; ++j) {
        base[j] = tot;
        tot += nx[j] * ny[j];
    }
    for (int i = threadIdx.x; i < g.nx * g.ny; i += blockDim.x) {
        const int yy = i / g.nx, xx = i - yy * g.nx;
        a[i] = A[g.off + (long long)yy * g.pitch + xx];
    }
    __syncthreads();
    for (int j = 1; j < J; ++j) {
        for (int i = threadIdx.x; i < nx[j] * ny[j]; i += blockDim.x) {
            const int yy = i / nx[j], xx = i - yy * nx[j];
            const T* u = a + base[j - 1];
            const int w = nx[j - 1];
            a[base[j] + i] = T(0.25) * ((u[2 * yy * w + 2 * xx] + u[2 * yy * w + 2 * xx + 1]) +
                                        (u[(2 * yy + 1) * w + 2 * xx] + u[(2 * yy + 1) * w + 2 * xx + 1]));
        }
        __syncthreads();
    }
    const int j = J - 1, cx = nx[j], cy = ny[j], n = cx * cy;
    const T bt = mg_bt<T>(S[s], g.lvl + j);
    T* rowk = fac + kMgCoarsePx;
    const int row = threadIdx.x >> 2, c0 = (threadIdx.x & 3) * kMgInvCols;
    T m[kMgInvCols];
    {
        // row `row` of the operator: a^2 + 4 beta~ on the diagonal, -beta~ per
        // periodic neighbour (coinciding neighbours accumulate)
        int nb[4] = {-1, -1, -1, -1};
        T dg = T(0);
        if (row < n) {
            const int yy = row / cx, xx = row - yy * cx;
            dg = a[base[j] + row] + T(4) * bt;
            nb[0] = yy * cx + wrap(xx - 1, cx);
            nb[1] = yy * cx + wrap(xx + 1, cx);
            nb[2] = wrap(yy - 1, cy) * cx + xx;
            nb[3] = wrap(yy + 1, cy) * cx + xx;
        }
#pragma unroll
        for (int t = 0; t < kMgInvCols; ++t) {
            const int jj = c0 + t;
            T v = T(0);
            if (row < n) {
                if (jj == row) v += dg;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (nb[k] == jj) v -= bt;
            } else if (jj == row) {
                v = T(1);
            }
            m[t] = v;
        }
    }
    for (int k = 0; k < n; ++k) {
        // column k (M[row][k] for every row; M[k][k] is the pivot)
#pragma unroll
        for (int t = 0; t < kMgInvCols; ++t)
            if (c0 + t == k) fac[row] = m[t];
        __syncthreads();
        const T f = fac[row];
        if (row == k) {
            const T inv = T(1) / fac[k];
#pragma unroll
            for (int t = 0; t < kMgInvCols; ++t) {
                m[t] = (c0 + t == k ? T(1) : m[t]) * inv;
                rowk[c0 + t] = m[t];
            }
        }
        __syncthreads();
        if (row != k) {
#pragma unroll
            for (int t = 0; t < kMgInvCols; ++t) m[t] = fma(-f, rowk[c0 + t], c0 + t == k ? T(0) : m[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < kMgInvCols; ++t) M[row][c0 + t] = m[t];
    __syncthreads();
    T* Q = Qinv + (long long)s * kMgCoarsePx * kMgCoarsePx;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
        const int i = q / n, jj = q - i * n;
        Q[q] = T(0.5) * (M[i][jj] + M[jj][i]);
    }
}

// The levels of one slice that fit one block (grid: one block per slice):
// f and a^2 of the slice's block level in, its correction e out.
template <typename T>
__global__ void __launch_bounds__(kMgBlockRunThreads)
    k_mg_block(const SliceGeom* GB, const SliceState* S, const T* F, const T* A, T* E, const T* Qinv,
               unsigned long long* acct) {
    extern __shared__ __align__(16) unsigned char mg_smem[];
    T* sh = reinterpret_cast<T*>(mg_smem);
    const int s = blockIdx.x;
    const SliceGeom g = GB[s];
    if (g.nx == 0 || !__ldg(&S[s].active) || __ldg(&S[s].cg_done)) return;
    int nx[kMgMaxBlockLevels], ny[kMgMaxBlockLevels], base[kMgMaxBlockLevels];
    const int J = mg_block_levels(g.nx, g.ny, nx, ny);
    int tot = 0;
    for (int j = 0; j < J; ++j) {
        base[j] = tot;
        tot += nx[j] * ny[j];
    }
    T* f = sh;             // f of every level
    T* a = sh + tot;       // a^2
    T* x = sh + 2 * tot;   // correction
    T* r = sh + 3 * tot;   // residual of a smoothing sweep (size of the first level)
    if (threadIdx.x == 0) atomicAdd(acct + KF_MG_BLOCK, (unsigned long long)(g.nx * g.ny) * 3ull * sizeof(T));
    const T om = mg_omega<T>();
    T bt[kMgMaxBlockLevels];
    bt[0] = mg_bt<T>(S[s], g.lvl);
    for (int j = 1; j < J; ++j) bt[j] = bt[j - 1] * T(0.25);
    for (int i = threadIdx.x; i < g.nx * g.ny; i += blockDim.x) {
        const int yy = i / g.nx, xx = i - yy * g.nx;
        const long long d = g.off + (long long)yy * g.pitch + xx;
        f[i] = F[d];
        a[i] = A[d];
    }
    __syncthreads();
    auto at = [&](const T* v, int j, int yy, int xx) -> T {
        return v[base[j] + wrap_near(yy, ny[j]) * nx[j] + wrap_near(xx, nx[j])];
    };
    auto mv = [&](const T* v, int j, int yy, int xx) -> T {   // (a^2 + bt L) v at a pixel of level j
        const T c = at(v, j, yy, xx);
        const T l = (T(4) * c - at(v, j, yy, xx - 1) - at(v, j, yy, xx + 1)) -
                    (at(v, j, yy - 1, xx) + at(v, j, yy + 1, xx));
        return at(a, j, yy, xx) * c + bt[j] * l;
    };
    for (int j = 1; j < J; ++j) {
        for (int i = threadIdx.x; i < nx[j] * ny[j]; i += blockDim.x) {
            const int yy = i / nx[j], xx = i - yy * nx[j];
            a[base[j] + i] = T(0.25) * ((at(a, j - 1, 2 * yy, 2 * xx) + at(a, j - 1, 2 * yy, 2 * xx + 1)) +
                                        (at(a, j - 1, 2 * yy + 1, 2 * xx) + at(a, j - 1, 2 * yy + 1, 2 * xx + 1)));
        }
        __syncthreads();
    }
    // kMgBlockSweeps damped Jacobi sweeps of level j from the current x
    auto sweeps = [&](int j, int n_sweeps) {
        const T b4 = T(4) * bt[j];
        for (int sw = 0; sw < n_sweeps; ++sw) {
            for (int i = threadIdx.x; i < nx[j] * ny[j]; i += blockDim.x) {
                const int yy = i / nx[j], xx = i - yy * nx[j];
                r[i] = f[base[j] + i] - mv(x, j, yy, xx);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nx[j] * ny[j]; i += blockDim.x)
                x[base[j] + i] += mg_div(om * r[i], a[base[j] + i] + b4);
            __syncthreads();
        }
    };
    // down: pre-smoothing from zero, restricted residual
    for (int j = 0; j + 1 < J; ++j) {
        const T b4 = T(4) * bt[j];
        for (int i = threadIdx.x; i < nx[j] * ny[j]; i += blockDim.x)
            x[base[j] + i] = mg_div(om * f[base[j] + i], a[base[j] + i] + b4);
        __syncthreads();
        sweeps(j, kMgBlockSweeps - 1);
        for (int i = threadIdx.x; i < nx[j + 1] * ny[j + 1]; i += blockDim.x) {
            const int yy = i / nx[j + 1], xx = i - yy * nx[j + 1];
            T sum = T(0);
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                    sum += at(f, j, 2 * yy + dy, 2 * xx + dx) - mv(x, j, 2 * yy + dy, 2 * xx + dx);
            f[base[j + 1] + i] = T(0.25) * sum;
        }
        __syncthreads();
    }
    // coarsest: exact solve with the inverse of its operator (symmetric, so
    // thread i reads column i, coalesced)
    {
        const int j = J - 1, n = nx[j] * ny[j];
        const T* Q = Qinv + (long long)s * kMgCoarsePx * kMgCoarsePx;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            T acc = T(0);
            for (int k = 0; k < n; ++k) acc = fma(Q[k * n + i], f[base[j] + k], acc);
            x[base[j] + i] = acc;
        }
        __syncthreads();
    }
    // up: coarse correction, post-smoothing
    for (int j = J - 2; j >= 0; --j) {
        for (int i = threadIdx.x; i < nx[j] * ny[j]; i += blockDim.x) {
            const int yy = i / nx[j], xx = i - yy * nx[j];
            x[base[j] + i] += x[base[j + 1] + (yy >> 1) * nx[j + 1] + (xx >> 1)];
        }
        __syncthreads();
        sweeps(j, kMgBlockSweeps);
    }
    for (int i = threadIdx.x; i < g.nx * g.ny; i += blockDim.x) {
        const int yy = i / g.nx, xx = i - yy * g.nx;
        E[g.off + (long long)yy * g.pitch + xx] = x[i];
    }
}

// --------------------------------------------------------------------------
// Sinogram-domain f updates (domain 1): conjugate gradients on
//   [alpha_k A^T A / gamma + c'_k + beta L] f_k = rhs_k
// preconditioned by (alpha_k + c'_k + beta K)^-1 applied by FFT (kinds 4, 5
// of the column pass, which also reduces r.y).  Fields: x = f_k, r = CG_R,
// y = CG_Y, p = CG_P0, q = CG_Q, A^T A p in CG_P1; A^T A f_k of the
// iterate (formed for the right-hand sides) in A2 (k = 0) or RHS_Z (k = 1).
// --------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void fcg_coeffs(const SliceConst& c, int k, T& al, T& cp) {
    al = kc<T>(c, k ? KC_SINO_AL1 : KC_SINO_AL0);
    cp = kc<T>(c, k ? KC_SINO_CP1 : KC_SINO_CP0);
}

// r = rhs - (alpha/gamma A^T A x + c' x + beta L x); |rhs|^2, |r|^2; start of the solve
template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_fcg_init(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                              SliceState* S, Ptrs<T> P, int k, int* pending) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, SW = TileDim<T>::SW;
    __shared__ __align__(16) T sm[1][TileDim<T>::TH + 2][SW];
    __shared__ double red[2 * 32];
    __shared__ SliceGeom s_g;
    const T* x = P.f[k ? RECON_F_F2 : RECON_F_F1];
    const T* gx = P.f[k ? RECON_F_RHS_Z : RECON_F_A2];
    const T* rhs = P.f[k ? RECON_F_RHS_F2 : RECON_F_RHS_F1];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        if (!__ldg(&S[it.slice].active)) continue;
        stage_struct(&s_g, G + it.slice);
        __syncthreads();
        const SliceGeom& g = s_g;
        account(P.acct, KF_FCG, tile_px<T>(g, it) * 4 * (long long)sizeof(T));
        load_tile<T, 1>(
            sm, g, it.a, it.b, [&](long long d) { return Vals<T, 1>{{x[d]}}; },
            [&](long long d) { return PVals<T, 1>{{ldv(x, d)}}; });
        __syncthreads();
        T al, cp;
        fcg_coeffs<T>(C[it.slice], k, al, cp);
        const T bt = Sc<T>::beta(S[it.slice]);
        T acc_b = T(0), acc_r = T(0);
        for_tile_vectors<T>(g, it, [&](long long d, int cnt, int ly, int lx0) {
            const Pack<T> gv = ldv_n(gx, d, cnt), b = ldv_n(rhs, d, cnt);
            Pack<T> r;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const T xc = sm[0][ly + 1][OFF + lx0 + e];
                r.v[e] = b.v[e] - (al * gv.v[e] + cp * xc + bt * lap5<T>(sm[0], ly + 1, OFF + lx0 + e));
                if (e < cnt) {
                    acc_b = fma(b.v[e], b.v[e], acc_b);
                    acc_r = fma(r.v[e], r.v[e], acc_r);
                }
            }
            stv_n(P.f[RECON_F_CG_R], d, r, cnt);
        });
        const T part[2] = {acc_b, acc_r};
        double acc[2];
        block_sum_t<T, 2>(part, acc, red);
        double tot[2];
        if (item_reduce<2>(L, w, it.slice, acc, tot, red)) {
            SliceState& so = S[it.slice];
            const double tol2 = C[it.slice].cg_tol * C[it.slice].cg_tol;
            so.bb = tot[0];
            so.rr = tot[1];
            so.rr0 = tot[1];
            so.cg_it = 0;
            so.ry = 0.0;
            set_betacg(so, 0.0);
            so.cg_done = (tot[0] == 0.0 || !(tot[1] > tol2 * tot[0])) ? 1 : 0;
            if (!so.cg_done) atomicAdd(pending, 1);
        }
        __syncthreads();
    }
}

// p = y + beta_cg p (p = y on the first step)
template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_fcg_p(ItemList L, const SliceGeom* G, const SliceState* S,
                                                           Ptrs<T> P) {
    constexpr int VN = TileDim<T>::VN;
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const SliceGeom g = G[it.slice];
        account(P.acct, KF_FCG, tile_px<T>(g, it) * 3 * (long long)sizeof(T));
        const bool first = __ldg(&sp->cg_it) == 0;
        const T bc = first ? T(0) : Sc<T>::betacg(*sp);
        for_tile_vectors<T>(g, it, [&](long long d, int cnt, int, int) {
            const Pack<T> y = ldv_n(P.f[RECON_F_CG_Y], d, cnt);
            Pack<T> p = first ? y : ldv_n(P.f[RECON_F_CG_P0], d, cnt);
            if (!first) {
#pragma unroll
                for (int e = 0; e < VN; ++e) p.v[e] = fma(bc, p.v[e], y.v[e]);
            }
            stv_n(P.f[RECON_F_CG_P0], d, p, cnt);
        });
    }
}

// q = alpha/gamma A^T A p + c' p + beta L p, p.q -> alpha
template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_fcg_q(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                           SliceState* S, Ptrs<T> P, int k) {
    constexpr int VN = TileDim<T>::VN, OFF = TileDim<T>::OFF, SW = TileDim<T>::SW;
    __shared__ __align__(16) T sm[1][TileDim<T>::TH + 2][SW];
    __shared__ double red[32];
    __shared__ SliceGeom s_g;
    const T* p = P.f[RECON_F_CG_P0];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        stage_struct(&s_g, G + it.slice);
        __syncthreads();
        const SliceGeom& g = s_g;
        account(P.acct, KF_FCG, tile_px<T>(g, it) * 3 * (long long)sizeof(T));
        load_tile<T, 1>(
            sm, g, it.a, it.b, [&](long long d) { return Vals<T, 1>{{p[d]}}; },
            [&](long long d) { return PVals<T, 1>{{ldv(p, d)}}; });
        __syncthreads();
        T al, cp;
        fcg_coeffs<T>(C[it.slice], k, al, cp);
        const T bt = Sc<T>::beta(*sp);
        T accT = T(0);
        for_tile_vectors<T>(g, it, [&](long long d, int cnt, int ly, int lx0) {
            const Pack<T> ap = ldv_n(P.f[RECON_F_CG_P1], d, cnt);
            Pack<T> q;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const T pc = sm[0][ly + 1][OFF + lx0 + e];
                q.v[e] = al * ap.v[e] + cp * pc + bt * lap5<T>(sm[0], ly + 1, OFF + lx0 + e);
                if (e < cnt) accT = fma(pc, q.v[e], accT);
            }
            stv_n(P.f[RECON_F_CG_Q], d, q, cnt);
        });
        const T part[1] = {accT};
        double acc[1];
        block_sum_t<T, 1>(part, acc, red);
        double tot[1];
        if (item_reduce<1>(L, w, it.slice, acc, tot, red)) {
            SliceState& so = S[it.slice];
            so.pq = tot[0];
            set_alpha(so, tot[0] > 0.0 ? so.ry / tot[0] : 0.0);
        }
        __syncthreads();
    }
}

// x += alpha p, r -= alpha q, r.r and the convergence test
template <typename T>
__global__ void __launch_bounds__(kStencilThreads) k_fcg_update(ItemList L, const SliceGeom* G, const SliceConst* C,
                                                                SliceState* S, Ptrs<T> P, int k, int* pending) {
    constexpr int VN = TileDim<T>::VN;
    __shared__ double red[32];
    T* x = P.f[k ? RECON_F_F2 : RECON_F_F1];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const SliceGeom g = G[it.slice];
        account(P.acct, KF_FCG, tile_px<T>(g, it) * 6 * (long long)sizeof(T));
        const T al = Sc<T>::alpha(*sp);
        T accT = T(0);
        for_tile_vectors<T>(g, it, [&](long long d, int cnt, int, int) {
            Pack<T> xv = ldv_n(x, d, cnt), r = ldv_n(P.f[RECON_F_CG_R], d, cnt);
            const Pack<T> pv = ldv_n(P.f[RECON_F_CG_P0], d, cnt), q = ldv_n(P.f[RECON_F_CG_Q], d, cnt);
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                xv.v[e] = fma(al, pv.v[e], xv.v[e]);
                r.v[e] = fma(-al, q.v[e], r.v[e]);
                if (e < cnt) accT = fma(r.v[e], r.v[e], accT);
            }
            stv_n(x, d, xv, cnt);
            stv_n(P.f[RECON_F_CG_R], d, r, cnt);
        });
        const T part[1] = {accT};
        double acc[1];
        block_sum_t<T, 1>(part, acc, red);
        double tot[1];
        if (item_reduce<1>(L, w, it.slice, acc, tot, red)) {
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

// sinogram combination of the data images: out = (a_k0 s_L + a_k1 s_H) / (S gamma)
__global__ void k_sino_combine(long long n, const float* sL, const float* sH, float wL, float wH, float* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = wL * sL[i] + wH * sH[i];
}

__global__ void k_next_beta(int n, const SliceConst* C, SliceState* S) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SliceState& st = S[s];
    if (!st.active) return;
    const SliceConst& c = C[s];
    st.k += 1;
    set_beta(st, st.beta * c.kappa, c);
    st.active = st.k < c.iters;
}

__global__ void k_reset_state(int n, const SliceConst* C, SliceState* S) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const SliceConst& c = C[s];
    SliceState st = {};
    set_beta(st, c.beta0, c);
    st.k = 0;
    st.active = c.iters > 0;
    st.cg_done = 1;
    S[s] = st;
}

// --------------------------------------------------------------------------
// Z = Z_w z^(1/m), z = Z^m / Z_w^m (Sec. II-D: Z is the m-th root of Z^m);
// Z = 1 where z <= 0.  Safeguarded FP64 Newton on phi(y) = m ln y - ln z,
// y <- y (1 - (m ln y - ln z) / m), from the FP32 root.  That start is within
// a few FP32 ulps (relative error e ~ 1e-7) and the step is quadratic (error
// about e^2 / 2), so one step reaches FP64 working accuracy, far below the
// rounding of the FP32 output.  Where z is outside the normal FP32 range the
// start is not that close, and the closed form exp(ln z / m) is taken.
// --------------------------------------------------------------------------

__device__ __forceinline__ double mth_root_newton(double z, double m, double inv_m) {
    const double lz = log(z);
    const float zf = (float)z;
    if (!(zf >= FLT_MIN) || isinf(zf)) return exp(lz * inv_m);
    const double y0 = (double)powf(zf, (float)inv_m);
    return y0 * (1.0 - (m * log(y0) - lz) * inv_m);
}

// The two-step comparator's maps of every slice from the loaded image pair:
// the initialisation (init_pixel) with rho_e and z rounded to the map
// precision as k_init stores them, then Z as k_extract forms it -- the maps
// recon_get returns right after recon_set_data -- into unpadded Z, rho_e,
// without touching the solve's state.  With lo, hi set, the image pair is read
// from those unpadded images (in 1/mm, normalised and rounded as k_load does)
// instead of the loaded fields; Z may alias lo and rhoe hi (each thread reads
// its pixel's pair before it writes that pixel).
template <typename T>
__global__ void k_direct(ItemList L, const SliceGeom* G, const SliceConst* C, Ptrs<T> P, const float* lo,
                         const float* hi, float* Z, float* rhoe, double zw, double m) {
    const double inv_m = 1.0 / m;
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceGeom g = G[it.slice];
        const SliceConst c = C[it.slice];
        for (int q = threadIdx.x; q < kTileW * TileH<T>::v; q += blockDim.x) {
            const int x = it.a + (q & (kTileW - 1)), y = it.b + q / kTileW;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const long long e = g.ext_off + (long long)y * g.nx + x;
            double f1, f2, rho, z;
            const T uL = lo ? T((double)lo[e] * c.inv_S) : P.f[RECON_F_MUL][d];
            const T uH = hi ? T((double)hi[e] * c.inv_S) : P.f[RECON_F_MUH][d];
            init_pixel(c, uL, uH, f1, f2, rho, z);
            const double zs = (double)T(z);
            Z[e] = zs > 0.0 ? (float)(zw * mth_root_newton(zs, m, inv_m)) : 1.0f;
            rhoe[e] = (float)T(rho);
        }
    }
}

// Monoenergetic images (eq. mac_E1/E2 at any energy): for energy k,
// out[k * n_ext + e] = f1 c[k][0] + f2 c[k][1] with c[k][j] = S mu_hat_j(E_k)
// of basis j (1/mm), from the current basis fractions, in the map precision.
constexpr int kMonoMax = 16;
struct MonoCoef {
    int n;
    double c[kMonoMax][2];
};

template <typename T>
__global__ void k_mono(ItemList L, const SliceGeom* G, Ptrs<T> P, MonoCoef mc, float* out, long long n_ext) {
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceGeom g = G[it.slice];
        for (int q = threadIdx.x; q < kTileW * TileH<T>::v; q += blockDim.x) {
            const int x = it.a + (q & (kTileW - 1)), y = it.b + q / kTileW;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const long long e = g.ext_off + (long long)y * g.nx + x;
            const T f1 = P.f[RECON_F_F1][d], f2 = P.f[RECON_F_F2][d];
            for (int k = 0; k < mc.n; ++k)
                out[k * n_ext + e] = (float)(f1 * T(mc.c[k][0]) + f2 * T(mc.c[k][1]));
        }
    }
}

template <typename T>
__global__ void k_extract(ItemList L, const SliceGeom* G, Ptrs<T> P, float* Z, float* rhoe, float* f1, float* f2,
                          double zw, double m) {
    const double inv_m = 1.0 / m;
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceGeom g = G[it.slice];
        for (int q = threadIdx.x; q < kTileW * TileH<T>::v; q += blockDim.x) {
            const int x = it.a + (q & (kTileW - 1)), y = it.b + q / kTileW;
            if (x >= g.nx || y >= g.ny) continue;
            const long long d = g.off + (long long)y * g.pitch + x;
            const long long e = g.ext_off + (long long)y * g.nx + x;
            if (Z) {
                const double z = P.f[RECON_F_Z][d];
                Z[e] = z > 0.0 ? (float)(zw * mth_root_newton(z, m, inv_m)) : 1.0f;
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
    p.sym = static_cast<const T*>(c.d_sym);
    return p;
}

int grid_for(const Ctx& c, int work) {
    const int cap = c.sm_count * c.grid_mult;
    return work < cap ? (work > 0 ? work : 1) : cap;
}

template <typename T>
int fft_smem_bytes(const Ctx& c) {
    int slots = 0;
    for (const SliceGeom& g : c.sg) {
        const int r = (g.rows_per_item + 1) * padded_len(g.nx);
        const int q = g.cols_per_item * col_ld(g.ny);
        slots = r > slots ? r : slots;
        slots = q > slots ? q : slots;
    }
    slots = (slots + 1) & ~1;   // the second buffer starts on a 16-byte boundary
    return 2 * slots * (int)sizeof(cplx<T>);
}

template <typename T>
int fft_half_slots(const Ctx& c) {
    return fft_smem_bytes<T>(c) / (2 * (int)sizeof(cplx<T>));
}

template <typename T>
int fft_solve(Ctx& c, const FftJobs& J) {
    const Ptrs<T> P = ptrs<T>(c);
    const int smem = fft_smem_bytes<T>(c);
    const cplx<T>* tw = static_cast<const cplx<T>*>(c.d_tw);
    const int half = fft_half_slots<T>(c);
    {
        FamTimer t(c, KF_ROWS_FWD);
        k_rows_fwd<T><<<grid_for(c, c.rows.n * J.n), kFftThreads, smem, c.stream>>>(c.rows.view(), c.d_geom,
                                                                                    c.d_state, P, J, tw, half);
    }
    {
        FamTimer t(c, KF_COLS);
        k_cols<T><<<grid_for(c, c.cols.n * J.n), kFftThreads, smem, c.stream>>>(c.cols.view(), c.d_geom, c.d_const,
                                                                               c.d_state, P, J, tw, half);
    }
    {
        FamTimer t(c, KF_ROWS_INV);
        k_rows_inv<T><<<grid_for(c, c.rows.n * J.n), kFftThreads, smem, c.stream>>>(c.rows.view(), c.d_geom,
                                                                                    c.d_state, P, J, tw, half);
    }
    c.launches += 3;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

int fft_item_slots(int nx, int ny, int budget);

template <typename T>
int set_fft_smem(Ctx& c) {
    int smem = fft_smem_bytes<T>(c);
    if (c.server_mode) {
        // a slot may later hold any 7-smooth size up to the capacity
        std::vector<int> sz;
        const int top = c.cap_nx > c.cap_ny ? c.cap_nx : c.cap_ny;
        for (int n = 1; n <= top; ++n) {
            int m = n;
            for (int f : {2, 3, 5, 7})
                while (m % f == 0) m /= f;
            if (m == 1) sz.push_back(n);
        }
        for (int nx : sz)
            for (int ny : sz)
                if (nx <= c.cap_nx && ny <= c.cap_ny) {
                    const int b = 2 * ((fft_item_slots(nx, ny, FftBudget<T>::E) + 1) & ~1) * (int)sizeof(cplx<T>);
                    smem = b > smem ? b : smem;
                }
    }
    RECON_CUDA(cudaFuncSetAttribute(k_rows_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_rows_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_pcg_fwd<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_pcg_fwd<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RECON_CUDA(cudaFuncSetAttribute(k_pcg_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
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
    if (stats) {
        k_thr_rhs<T, true><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom,
                                                                                     c.d_const, c.d_state, P);
        c.launches += 1;
    } else {
        // FP32 slices up to kBandMaxW wide on the band kernel, the others on tiles
        if constexpr (std::is_same<T, float>::value) {
            const DevItemList& B = c.thr_band;
            if (B.n) {
                if (c.domain != 0)
                    k_thr_band<true><<<grid_for(c, B.n), kStripThreads, band_smem_bytes<8>(), c.stream>>>(
                        B.view(), c.d_geom, c.d_const, c.d_state, P, kThrRows);
                else
                    k_thr_band<false><<<grid_for(c, B.n), kStripThreads, band_smem_bytes<6>(), c.stream>>>(
                        B.view(), c.d_geom, c.d_const, c.d_state, P, kThrRows);
                c.launches += 1;
            }
        }
        const DevItemList& L = std::is_same<T, float>::value ? c.thr_tiles : c.tiles;
        if (L.n) {
            k_thr_rhs<T, false><<<grid_for(c, L.n), kStencilThreads, 0, c.stream>>>(L.view(), c.d_geom, c.d_const,
                                                                                   c.d_state, P);
            c.launches += 1;
        }
    }
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
        return fft_solve<T>(c, J);
    }
    if ((rc = fft_solve<T>(c, jobs1(RECON_F_RHS_F1, 0, RECON_F_F1, 0)))) return rc;
    k_gs_fix<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, c.d_const,
                                                                         c.d_state, ptrs<T>(c));
    c.launches += 1;
    return fft_solve<T>(c, jobs1(RECON_F_RHS_F2, 1, RECON_F_F2, 1));
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

// Family timer that is skipped while a graph is captured.
struct MaybeTimer {
    std::unique_ptr<FamTimer> t;
    MaybeTimer(Ctx& c, int fam, bool on) {
        if (on) t.reset(new FamTimer(c, fam));
    }
};

template <typename T>
T* field_t(Ctx& c, int f) {
    return static_cast<T*>(c.field[f]);
}

// Residual buffer k of the multigrid PCG (its steps alternate between two).
template <typename T>
T* mg_r(Ctx& c, int k) {
    return field_t<T>(c, k ? RECON_F_CG_R2 : RECON_F_CG_R);
}

// Rows a warp walks per strip item on multigrid level l: mg_rb on the fine
// level; on a coarse level the count level_items chose for the handle's
// items, else mg_rb halved per level (grids of a quarter of the pixels), at
// least 8.
int strip_rows(const Ctx& c, int l) {
    if (l >= 1 && l < (int)c.mg_level_rb.size() && c.mg_level_rb[l] > 0) return c.mg_level_rb[l];
    const int r = c.mg_rb >> l;
    return r < 8 ? 8 : r;
}

// One pass of the strip family on level l: the band kernel over the band items
// (levels up to kBandMaxW wide), the ghost-column strip kernel over the strip
// items of wider levels.
template <typename FB, typename FS>
void strip_pass(Ctx& c, int l, FB band, FS wide, bool with_band = true) {
    if (with_band && c.mg_strips[l].n) {
        band(c.mg_strips[l]);
        c.launches += 1;
    }
    if (c.mg_wide[l].n) {
        wide(c.mg_wide[l]);
        c.launches += 1;
    }
}

// a^2 of every multigrid level from the fine a^2 (once per Z^m solve).
template <typename T>
void mg_restrict_a2(Ctx& c, bool timed) {
    MaybeTimer t(c, KF_MG_SETUP, timed);
    T* pa = static_cast<T*>(c.mg_pool[1]);
    // levels 1 .. F in one pass over the fine tiles (F = the tile's halvings), deeper levels one launch each
    constexpr int FT = ilog2c(TileDim<T>::TH);   // halvings of the tile height: 5 (FP32), 4 (FP64)
    static_assert(FT <= kMgRestrictFused, "level table too small");
    const int F = c.mg_max_lb < FT ? c.mg_max_lb : FT;
    if (F > 0) {
        MgLevelGeoms LG{};
        for (int l = 0; l <= F; ++l) LG.g[l] = c.d_mg_geom[l];
        const DevItemList& L = c.mg_tiles[0];
        k_mg_restrict_all<T><<<grid_for(c, L.n), kStencilThreads, 0, c.stream>>>(
            L.view(), LG, F, c.d_state, field_t<T>(c, RECON_F_A2), pa, c.d_acct);
        c.launches += 1;
    }
    for (int l = F; l < c.mg_max_lb; ++l) {
        const DevItemList& L = c.mg_tiles[l];
        const T* a = l == 0 ? field_t<T>(c, RECON_F_A2) : pa;
        k_mg_restrict<T><<<grid_for(c, L.n), kStencilThreads, 0, c.stream>>>(L.view(), c.d_mg_geom[l],
                                                                             c.d_mg_geom[l + 1], c.d_state, a, pa,
                                                                             c.d_acct);
        c.launches += 1;
    }
    k_mg_coarse_inv<T><<<c.n, kMgBlockThreads, c.mg_inv_smem, c.stream>>>(c.d_mg_block, c.d_state, pa,
                                                                          static_cast<T*>(c.mg_qinv));
    c.launches += 1;
}

// Fine-level start of a multigrid PCG step: UPD updates z and r (from
// residual buffer rk into buffer rk ^ 1) and tests convergence.
template <typename T, bool UPD>
void mg_fwd(Ctx& c, int par, int rk, bool timed) {
    MaybeTimer t(c, KF_MG_FWD, timed);
    if constexpr (std::is_same<T, float>::value) {
        // FP32: the register-streaming band / strip kernels over the fine level
        // (the first step of the band slices is part of k_mgb_start)
        const int rb = strip_rows(c, 0);
        strip_pass(
            c, 0,
            [&](const DevItemList& S) {
                k_mgb_fwd<UPD><<<grid_for(c, S.n), kStripThreads, band_smem_bytes<4>(), c.stream>>>(
                    S.view(), c.d_geom, c.d_mg_geom[1], c.d_const, c.d_state, ptrs<T>(c), par, mg_r<T>(c, rk),
                    mg_r<T>(c, rk ^ 1), field_t<T>(c, RECON_F_A2), static_cast<T*>(c.mg_pool[0]), c.d_cg_pending, rb,
                    0);
            },
            [&](const DevItemList& S) {
                k_mgs_fwd<UPD><<<grid_for(c, S.n), kStripThreads, strip_smem_bytes<4>(), c.stream>>>(
                    S.view(), c.d_geom, c.d_mg_geom[1], c.d_const, c.d_state, ptrs<T>(c), par, mg_r<T>(c, rk),
                    mg_r<T>(c, rk ^ 1), field_t<T>(c, RECON_F_A2), static_cast<T*>(c.mg_pool[0]), c.d_cg_pending, rb,
                    0);
            },
            UPD);
    } else {
        const DevItemList& L = c.mg_tiles[0];
        k_mg_fwd<T, UPD><<<grid_for(c, L.n), kStencilThreads, 2 * sizeof(MgBufFwd<T>), c.stream>>>(
            L.view(), c.d_geom, c.d_mg_geom[1], c.d_const, c.d_state, ptrs<T>(c), par, mg_r<T>(c, rk),
            mg_r<T>(c, rk ^ 1), static_cast<T*>(c.mg_pool[0]), c.d_cg_pending);
        c.launches += 1;
    }
}

// Fine level of the cycle and the new direction: y (k_mgs_y / k_mg_y), then p
// and p.q (k_mgs_pq / k_mg_pq).
template <typename T>
void mg_fine_tail(Ctx& c, int par, int rk, bool timed) {
    T* pe = static_cast<T*>(c.mg_pool[2]);
    if constexpr (std::is_same<T, float>::value) {
        const int rb = strip_rows(c, 0);
        {
            MaybeTimer t(c, KF_MG_Y, timed);
            strip_pass(
                c, 0,
                [&](const DevItemList& S) {
                    k_mgb_up<true><<<grid_for(c, S.n), kStripThreads, band_smem_bytes<3>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_mg_geom[1], c.d_state, ptrs<T>(c), mg_r<T>(c, rk),
                        field_t<T>(c, RECON_F_A2), pe, field_t<T>(c, RECON_F_CG_Y), rb, 0);
                },
                [&](const DevItemList& S) {
                    k_mgs_up<true><<<grid_for(c, S.n), kStripThreads, strip_smem_bytes<3>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_mg_geom[1], c.d_state, ptrs<T>(c), mg_r<T>(c, rk),
                        field_t<T>(c, RECON_F_A2), pe, field_t<T>(c, RECON_F_CG_Y), rb, 0);
                });
        }
        {
            MaybeTimer t(c, KF_MG_PQ, timed);
            strip_pass(
                c, 0,
                [&](const DevItemList& S) {
                    k_mgb_pq<false><<<grid_for(c, S.n), kStripThreads, band_smem_bytes<3>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_state, ptrs<T>(c), par, rb);
                },
                [&](const DevItemList& S) {
                    k_mgs_pq<false><<<grid_for(c, S.n), kStripThreads, strip_smem_bytes<3>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_state, ptrs<T>(c), par, rb);
                });
        }
    } else {
        const DevItemList& L0 = c.mg_tiles[0];
        {
            MaybeTimer t(c, KF_MG_Y, timed);
            k_mg_y<T><<<grid_for(c, L0.n), kStencilThreads, 2 * sizeof(MgBufHalo2<T>), c.stream>>>(
                L0.view(), c.d_geom, c.d_mg_geom[1], c.d_state, ptrs<T>(c), mg_r<T>(c, rk), pe);
        }
        {
            MaybeTimer t(c, KF_MG_PQ, timed);
            k_mg_pq<T><<<grid_for(c, L0.n), kStencilThreads, 2 * sizeof(MgBufPq<T>), c.stream>>>(
                L0.view(), c.d_geom, c.d_state, ptrs<T>(c), par);
        }
        c.launches += 2;
    }
}

// Rest of a multigrid PCG step for residual buffer rk: the V-cycle below the
// fine level, y and r.y, then p, q and p.q.
template <typename T>
void mg_tail(Ctx& c, int par, int rk, bool timed) {
    T* pf = static_cast<T*>(c.mg_pool[0]);
    T* pa = static_cast<T*>(c.mg_pool[1]);
    T* pe = static_cast<T*>(c.mg_pool[2]);
    {
        MaybeTimer t(c, KF_MG_LEVELS, timed);
        for (int l = 1; l < c.mg_max_lb; ++l) {
            if constexpr (std::is_same<T, float>::value) {
                const int rb = strip_rows(c, l);
                strip_pass(
                    c, l,
                    [&](const DevItemList& S) {
                        k_mgb_fwd<false><<<grid_for(c, S.n), kStripThreads, band_smem_bytes<4>(), c.stream>>>(
                            S.view(), c.d_mg_geom[l], c.d_mg_geom[l + 1], c.d_const, c.d_state, ptrs<T>(c), 0, pf,
                            nullptr, pa, pf, c.d_cg_pending, rb, l);
                    },
                    [&](const DevItemList& S) {
                        k_mgs_fwd<false><<<grid_for(c, S.n), kStripThreads, strip_smem_bytes<4>(), c.stream>>>(
                            S.view(), c.d_mg_geom[l], c.d_mg_geom[l + 1], c.d_const, c.d_state, ptrs<T>(c), 0, pf,
                            nullptr, pa, pf, c.d_cg_pending, rb, l);
                    });
            }
            const DevItemList& L = c.mg_tiles_rest[l];
            if (L.n) {
                k_mg_down<T><<<grid_for(c, L.n), kStencilThreads, 2 * sizeof(MgBufHalo2<T>), c.stream>>>(
                    L.view(), c.d_mg_geom[l], c.d_mg_geom[l + 1], c.d_state, pf, pa, pf, c.d_acct);
                c.launches += 1;
            }
        }
    }
    {
        MaybeTimer t(c, KF_MG_BLOCK, timed);
        k_mg_block<T><<<c.n, kMgBlockRunThreads, c.mg_block_smem, c.stream>>>(
            c.d_mg_block, c.d_state, pf, pa, pe, static_cast<const T*>(c.mg_qinv), c.d_acct);
        c.launches += 1;
    }
    {
        MaybeTimer t(c, KF_MG_LEVELS, timed);
        for (int l = c.mg_max_lb - 1; l >= 1; --l) {
            if constexpr (std::is_same<T, float>::value) {
                const int rb = strip_rows(c, l);
                strip_pass(
                    c, l,
                    [&](const DevItemList& S) {
                        k_mgb_up<false><<<grid_for(c, S.n), kStripThreads, band_smem_bytes<3>(), c.stream>>>(
                            S.view(), c.d_mg_geom[l], c.d_mg_geom[l + 1], c.d_state, ptrs<T>(c), pf, pa, pe, pe, rb,
                            l);
                    },
                    [&](const DevItemList& S) {
                        k_mgs_up<false><<<grid_for(c, S.n), kStripThreads, strip_smem_bytes<3>(), c.stream>>>(
                            S.view(), c.d_mg_geom[l], c.d_mg_geom[l + 1], c.d_state, ptrs<T>(c), pf, pa, pe, pe, rb,
                            l);
                    });
            }
            const DevItemList& L = c.mg_tiles_rest[l];
            if (L.n) {
                k_mg_up<T><<<grid_for(c, L.n), kStencilThreads, 2 * sizeof(MgBufHalo2<T>), c.stream>>>(
                    L.view(), c.d_mg_geom[l], c.d_mg_geom[l + 1], c.d_state, pf, pa, pe, pe, c.d_acct);
                c.launches += 1;
            }
        }
    }
    mg_fine_tail<T>(c, par, rk, timed);
}

// Start of a Z^m solve: the pending count cleared, r = rhs - M z and the PCG
// scalars of every slice (k_cg_init), and on the FP32 band slices also the
// first multigrid step (k_mgb_start does both there).
template <typename T>
void pcg_begin(Ctx& c, bool timed) {
    const Ptrs<T> P = ptrs<T>(c);
    cudaMemsetAsync(c.d_cg_pending, 0, 2 * sizeof(int), c.stream);
    MaybeTimer t0(c, KF_CG_INIT, timed);
    const DevItemList& ct = c.mg_max_lb > 0 ? c.cg_tiles : c.tiles;
    if (ct.n) {
        k_cg_init<T><<<grid_for(c, ct.n), kStencilThreads, 2 * sizeof(CgInitBuf<T>), c.stream>>>(
            ct.view(), c.d_geom, c.d_const, c.d_state, P, c.d_cg_pending);
        c.launches += 1;
    }
    if constexpr (std::is_same<T, float>::value) {
        const DevItemList& S = c.mg_max_lb > 0 ? c.mg_strips[0] : c.tiles;
        if (c.mg_max_lb > 0 && S.n) {
            k_mgb_start<<<grid_for(c, S.n), kStripThreads, band_smem_bytes<3>(), c.stream>>>(
                S.view(), c.d_geom, c.d_mg_geom[1], c.d_const, c.d_state, P, static_cast<float*>(c.mg_pool[0]),
                c.d_cg_pending, strip_rows(c, 0));
            c.launches += 1;
        }
    }
}

template <typename T>
int op_solve_z(Ctx& c) {
    const Ptrs<T> P = ptrs<T>(c);
    pcg_begin<T>(c, true);
    // slices on the FFT preconditioner (the row and column items of the PCG)
    // and slices on the multigrid cycle run side by side, step by step
    const bool mg = c.mg_max_lb > 0;
    const DevItemList& prow = mg ? c.pcg_rows : c.rows;
    const DevItemList& pcol = mg ? c.pcg_cols : c.cols;
    const bool fft = prow.n > 0;
    const int smem = fft_smem_bytes<T>(c);
    const cplx<T>* tw = static_cast<const cplx<T>*>(c.d_tw);
    const int half = fft_half_slots<T>(c);
    const FftJobs pre = jobs1(RECON_F_CG_R, 0, RECON_F_CG_Y, 3);
    int par = c.cg_parity;
    int rk = 0;   // multigrid residual buffer (k_cg_init wrote CG_R)
    // Consecutive FFT passes walk the items in opposite orders, so that each
    // pass starts on the slices the previous one touched last, which are
    // still in the L2 (the working set is many times the L2).  k_cg_init ran
    // forward, so the first PCG pass runs backward.
    int rev = 1;
    if (fft) {
        FamTimer t(c, KF_PCG_FWD);
        k_pcg_fwd<T, false><<<grid_for(c, prow.n), kFftThreads, smem, c.stream>>>(
            prow.view(), c.d_geom, c.d_const, c.d_state, P, tw, half, par, c.d_cg_pending, rev);
        rev ^= 1;
        c.launches += 1;
    }
    if (mg) {
        mg_restrict_a2<T>(c, true);
        mg_fwd<T, false>(c, par, rk, true);
    }
    int cap = 0;
    for (const auto& p : c.prm) cap = p.cg_max_iters > cap ? p.cg_max_iters : cap;
    // The host learns that every slice has converged by reading the pending
    // count, which costs a synchronisation.  The first read comes after as
    // many steps as the previous Z^m solve took (its slowest slice; the warm
    // started solves of consecutive iterations take similar counts), then
    // every two steps.
    const int first_check = c.cg_pred > 0 ? c.cg_pred : 4;
    for (int it = 0; it < cap; ++it) {
        if (fft) {
            {
                FamTimer t(c, KF_COLS_PRE);
                k_cols<T><<<grid_for(c, pcol.n), kFftThreads, smem, c.stream>>>(pcol.view(), c.d_geom, c.d_const,
                                                                                c.d_state, P, pre, tw, half, rev);
                rev ^= 1;
            }
            {
                FamTimer t(c, KF_PCG_INV);
                k_pcg_inv<T><<<grid_for(c, prow.n), kFftThreads, smem, c.stream>>>(prow.view(), c.d_geom, c.d_state,
                                                                                  P, tw, half, par, rev);
                rev ^= 1;
            }
            c.launches += 2;
        }
        if (mg) mg_tail<T>(c, par, rk, true);
        if (fft) {
            FamTimer t(c, KF_PCG_FWD);
            k_pcg_fwd<T, true><<<grid_for(c, prow.n), kFftThreads, smem, c.stream>>>(
                prow.view(), c.d_geom, c.d_const, c.d_state, P, tw, half, par, c.d_cg_pending, rev);
            rev ^= 1;
            c.launches += 1;
        }
        if (mg) {
            mg_fwd<T, true>(c, par, rk, true);
            rk ^= 1;
        }
        RECON_CUDA(cudaGetLastError());
        par ^= 1;
        const int done = it + 1;   // updating steps launched
        if ((done >= first_check && (done - first_check) % 2 == 0) || it == cap - 1) {
            RECON_CUDA(cudaMemcpyAsync(c.h_cg_pending, c.d_cg_pending, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                       c.stream));
            RECON_CUDA(cudaStreamSynchronize(c.stream));
            if (c.h_cg_pending[0] <= 0) {
                c.cg_pred = c.h_cg_pending[1];
                break;
            }
        }
    }
    c.cg_parity = par;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

// ---- sinogram-domain f updates (domain 1; FP32 fields) ----

// Slice s of a field: all slices of a domain-1 handle share one geometry, so
// they sit ny * pitch elements apart.
template <typename T>
T* field_base(Ctx& c, int f) {
    return static_cast<T*>(c.field[f]) + c.sg[0].off;
}

// out (cleared) = A^T A x over all slices.  Algorithmic HBM bytes: the image
// read and the sinogram written by A, the sinogram read and the image added
// to by A^T (the gathers themselves hit the L2-resident image).
int gram_all(Ctx& c, const float* x, float* out, const float* wt = nullptr) {
    const recon_geometry& g = c.geo[0];
    const long long pitch = c.sg[0].pitch, stride = (long long)c.sg[0].ny * pitch;
    FamTimer t(c, KF_PROJ);
    c.host_acct[KF_PROJ] += 4ull * (unsigned long long)c.n *
                            (3ull * g.nx * g.ny + (wt ? 3ull : 2ull) * (unsigned long long)g.n_views * g.n_bins);
    int rc;
    if ((rc = ct_project_pitched(g, c.n, x, pitch, stride, c.d_sino_tmp, c.stream, &c.launches))) return rc;
    RECON_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * stride * c.n, c.stream));
    return ct_backproject_add(g, c.n, c.d_sino_tmp, out, pitch, stride, c.stream, &c.launches, wt);
}

// ---- domain 2: polyenergetic sinogram fidelity linearised by Gauss-Newton ----
//
// Per ray of every slice, at l = (A f1, A f2) of the iterate (Jacobi, reading
// R1): the polyenergetic -log h_i(l) = -ln sum_b w_ib exp(-S (mu_1b l1 +
// mu_2b l2)) / S of each arm (w_ib its normalised detected spectrum; the
// photoelectric / Compton model is spanned by the two basis materials at every
// energy, Sec. II-B), its derivatives J_ik = sum_b om_ib mu_kb (om: the
// spectrum reweighted by the ray's attenuation), d_i = s_i / S - h_i + J_i1 l1
// + J_i2 l2, W_kl = sum_i J_ik J_il and v_k = sum_i J_ik d_i - W_ko l_o.  The
// f_k normal equations become [A^T diag(W_kk) A / gamma + c'_k + beta L] f_k
// = A^T v_k / gamma + (model terms) + beta div(h, v): the linear mode's with
// per-ray weights.  Sums over the bins start from the smallest exponent, so
// no term underflows.
constexpr int kGnArrays = 6;   // per ray: l1, l2, W11, W22, v1 / gamma, v2 / gamma
__global__ void k_gn_rays(long long n_rays, const float* __restrict__ sL, const float* __restrict__ sH,
                          const float* __restrict__ spec, int nb0, int nb1, float S, float inv_gamma, float* gn) {
    extern __shared__ float tab[];   // (nb0 + nb1) x (w, mu_hat_1, mu_hat_2)
    for (int i = threadIdx.x; i < 3 * (nb0 + nb1); i += blockDim.x) tab[i] = spec[i];
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const float l1 = gn[r], l2 = gn[n_rays + r];
    float W11 = 0.f, W22 = 0.f, W12 = 0.f, u1 = 0.f, u2 = 0.f;
    for (int arm = 0; arm < 2; ++arm) {
        const float* t = tab + (arm ? 3 * nb0 : 0);
        const int nb = arm ? nb1 : nb0;
        float tmin = INFINITY;
        for (int b = 0; b < nb; ++b) tmin = fminf(tmin, fmaf(t[3 * b + 1], l1, t[3 * b + 2] * l2));
        float se = 0.f, s1 = 0.f, s2 = 0.f;
        for (int b = 0; b < nb; ++b) {
            const float m1 = t[3 * b + 1], m2 = t[3 * b + 2];
            const float e = t[3 * b] * expf(-S * (fmaf(m1, l1, m2 * l2) - tmin));
            se += e;
            s1 = fmaf(e, m1, s1);
            s2 = fmaf(e, m2, s2);
        }
        const float J1 = s1 / se, J2 = s2 / se;
        const float h = tmin - logf(se) / S;
        const float d = (arm ? sH : sL)[r] / S - h + fmaf(J1, l1, J2 * l2);
        W11 = fmaf(J1, J1, W11);
        W22 = fmaf(J2, J2, W22);
        W12 = fmaf(J1, J2, W12);
        u1 = fmaf(J1, d, u1);
        u2 = fmaf(J2, d, u2);
    }
    gn[2 * n_rays + r] = W11;
    gn[3 * n_rays + r] = W22;
    gn[4 * n_rays + r] = (u1 - W12 * l2) * inv_gamma;
    gn[5 * n_rays + r] = (u2 - W12 * l1) * inv_gamma;
}

// The Gauss-Newton terms of the iterate: t_k = A^T v_k / gamma into MUL (k = 0)
// and MUH (k = 1), the weighted Gram images A^T (W_kk o A f_k) into A2 and
// RHS_Z (read by the right-hand sides and by the starts of the two CG solves).
int op_gn_terms(Ctx& c) {
    const recon_geometry& g = c.geo[0];
    const long long nr = (long long)g.n_views * g.n_bins, n_rays = nr * c.n;
    const long long pitch = c.sg[0].pitch, stride = (long long)c.sg[0].ny * pitch;
    FamTimer t(c, KF_PROJ);
    c.host_acct[KF_PROJ] += 4ull * (unsigned long long)c.n *
                            (6ull * g.nx * g.ny + 18ull * (unsigned long long)nr);
    int rc;
    float* l1 = c.d_gn;
    float* l2 = c.d_gn + n_rays;
    if ((rc = ct_project_pitched(g, c.n, field_base<float>(c, RECON_F_F1), pitch, stride, l1, c.stream,
                                 &c.launches)))
        return rc;
    if ((rc = ct_project_pitched(g, c.n, field_base<float>(c, RECON_F_F2), pitch, stride, l2, c.stream,
                                 &c.launches)))
        return rc;
    const int smem = 3 * (c.spec_nb[0] + c.spec_nb[1]) * (int)sizeof(float);
    k_gn_rays<<<(unsigned)((n_rays + 255) / 256), 256, smem, c.stream>>>(
        n_rays, c.d_sino[0], c.d_sino[1], c.d_spec, c.spec_nb[0], c.spec_nb[1], (float)scale_per_mm(),
        (float)c.hconst[0].inv_gamma, c.d_gn);
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    const int out[4] = {RECON_F_MUL, RECON_F_MUH, RECON_F_A2, RECON_F_RHS_Z};
    const float* src[4] = {c.d_gn + 4 * n_rays, c.d_gn + 5 * n_rays, l1, l2};
    const float* wt[4] = {nullptr, nullptr, c.d_gn + 2 * n_rays, c.d_gn + 3 * n_rays};
    for (int k = 0; k < 4; ++k) {
        float* o = field_base<float>(c, out[k]);
        RECON_CUDA(cudaMemsetAsync(o, 0, sizeof(float) * stride * c.n, c.stream));
        if ((rc = ct_backproject_add(g, c.n, src[k], o, pitch, stride, c.stream, &c.launches, wt[k]))) return rc;
    }
    return RECON_OK;
}

// A^T A f1 into A2 and A^T A f2 into RHS_Z (read by the right-hand sides
// and by the starts of the two CG solves; the synthesis rewrites both)
template <typename T>
int op_modeb_gram(Ctx& c) {
    if constexpr (std::is_same<T, float>::value) {
        int rc;
        if ((rc = gram_all(c, field_base<float>(c, RECON_F_F1), field_base<float>(c, RECON_F_A2)))) return rc;
        return gram_all(c, field_base<float>(c, RECON_F_F2), field_base<float>(c, RECON_F_RHS_Z));
    } else {
        set_error("domain 1 needs precision 1");
        return RECON_EINVAL;
    }
}

template <typename T>
int op_solve_f_sino(Ctx& c) {
    if constexpr (!std::is_same<T, float>::value) {
        set_error("domain 1 needs precision 1");
        return RECON_EINVAL;
    } else {
        const Ptrs<T> P = ptrs<T>(c);
        int cap = 0;
        for (const auto& p : c.prm) cap = p.cg_max_iters > cap ? p.cg_max_iters : cap;
        int rc;
        for (int k = 0; k < 2; ++k) {
            const FftJobs pre = jobs1(RECON_F_CG_R, 0, RECON_F_CG_Y, 4 + k);
            RECON_CUDA(cudaMemsetAsync(c.d_cg_pending, 0, sizeof(int), c.stream));
            {
                FamTimer t(c, KF_FCG);
                k_fcg_init<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(
                    c.tiles.view(), c.d_geom, c.d_const, c.d_state, P, k, c.d_cg_pending);
            }
            c.launches += 1;
            if ((rc = fft_solve<T>(c, pre))) return rc;
            for (int it = 0; it < cap; ++it) {
                {
                    FamTimer t(c, KF_FCG);
                    k_fcg_p<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom,
                                                                                        c.d_state, P);
                }
                const float* wt = c.domain == 2 ? c.d_gn + (long long)(2 + k) * c.n * c.geo[0].n_views * c.geo[0].n_bins
                                                : nullptr;
                if ((rc = gram_all(c, field_base<float>(c, RECON_F_CG_P0), field_base<float>(c, RECON_F_CG_P1), wt)))
                    return rc;
                {
                    FamTimer t(c, KF_FCG);
                    k_fcg_q<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(
                        c.tiles.view(), c.d_geom, c.d_const, c.d_state, P, k);
                    k_fcg_update<T><<<grid_for(c, c.tiles.n), kStencilThreads, 0, c.stream>>>(
                        c.tiles.view(), c.d_geom, c.d_const, c.d_state, P, k, c.d_cg_pending);
                }
                c.launches += 3;
                RECON_CUDA(cudaGetLastError());
                if ((rc = fft_solve<T>(c, pre))) return rc;
                if ((it & 3) == 3 || it == cap - 1) {
                    RECON_CUDA(cudaMemcpyAsync(c.h_cg_pending, c.d_cg_pending, sizeof(int), cudaMemcpyDeviceToHost,
                                               c.stream));
                    RECON_CUDA(cudaStreamSynchronize(c.stream));
                    if (*c.h_cg_pending <= 0) break;
                }
            }
        }
        return RECON_OK;
    }
}

template <typename T>
int op_next_beta(Ctx& c) {
    k_next_beta<<<(c.n + 127) / 128, 128, 0, c.stream>>>(c.n, c.d_const, c.d_state);
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

int alloc_dev(Ctx& c, void** p, size_t bytes);

// ---- one iteration as a CUDA graph ----

// Set the WHILE condition of the PCG loop before its first body.
__global__ void k_pcg_loop_start(cudaGraphConditionalHandle h, const int* pending, int* body) {
    *body = 0;
    cudaGraphSetConditional(h, *pending > 0 ? 1u : 0u);
}

// End of a body (two PCG steps): run another while a slice has not
// converged and fewer than `cap` bodies have run (bounded loop).
__global__ void k_pcg_loop_cond(cudaGraphConditionalHandle h, const int* pending, int* body, int cap,
                                unsigned long long* launches, int per_body) {
    const int b = *body + 1;
    *body = b;
    cudaGraphSetConditional(h, (*pending > 0 && b < cap) ? 1u : 0u);
    atomicAdd(launches, (unsigned long long)per_body);   // the body's PCG kernels and this one
}

template <typename T>
int graph_build_t(Ctx& c) {
    const Ptrs<T> P = ptrs<T>(c);
    const int smem = fft_smem_bytes<T>(c), smem_c = smem;
    const cplx<T>* tw = static_cast<const cplx<T>*>(c.d_tw);
    const int half = fft_half_slots<T>(c), half_c = half;
    const FftJobs pre = jobs1(RECON_F_CG_R, 0, RECON_F_CG_Y, 3);
    const bool mg = c.mg_max_lb > 0;
    const DevItemList& prow = mg ? c.pcg_rows : c.rows;
    const DevItemList& pcol = mg ? c.pcg_cols : c.cols;
    const bool fft = prow.n > 0;
    int cap = 0;
    for (const auto& p : c.prm) cap = p.cg_max_iters > cap ? p.cg_max_iters : cap;
    const int bodies = (cap + 1) / 2;
    cudaStream_t user = c.stream;
    c.stream = c.graph_stream;   // the op functions launch on c.stream
    int rc = RECON_OK;
    const long long l0 = c.launches;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t cond = nullptr;
    auto fail = [&](cudaError_t e, const char* what) {
        c.stream = user;
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, what);
    };
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return fail(e, "cudaGraphCreate");
    e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail(e, "cudaGraphConditionalHandleCreate");
    // 1. threshold + rhs, f and rho_e solves, synthesis, start of the PCG
    e = cudaStreamBeginCaptureToGraph(c.stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e, "capture (iteration head)");
    if (!rc) rc = op_thr_rhs<T>(c, false);
    if (!rc) rc = op_solve_f<T>(c);
    if (!rc) rc = op_synth<T>(c);
    if (!rc) rc = fft_solve<T>(c, jobs1(RECON_F_RHS_RHO, 2, RECON_F_RHO, 2));
    if (!rc) {
        pcg_begin<T>(c, false);
        if (fft) {
            k_pcg_fwd<T, false><<<grid_for(c, prow.n), kFftThreads, smem, c.stream>>>(
                prow.view(), c.d_geom, c.d_const, c.d_state, P, tw, half, 0, c.d_cg_pending, 1);
            c.launches += 1;
        }
        if (mg) {
            mg_restrict_a2<T>(c, false);
            mg_fwd<T, false>(c, 0, 0, false);
        }
        k_pcg_loop_start<<<1, 1, 0, c.stream>>>(h, c.d_cg_pending, c.d_graph_body);
        c.launches += 1;
    }
    e = cudaStreamEndCapture(c.stream, &g);
    if (rc) {
        c.stream = user;
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(e, "capture end (iteration head)");
    // leaves of the head become the dependencies of the loop
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn), leaves;
    cudaGraphGetNodes(g, nodes.data(), &nn);
    for (cudaGraphNode_t n : nodes) {
        size_t nd = 0;
        cudaGraphNodeGetDependentNodes(n, nullptr, nullptr, &nd);
        if (nd == 0) leaves.push_back(n);
    }
    // 2. WHILE (pending && body < bodies): two PCG steps
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cond, g, leaves.data(), nullptr, leaves.size(), &cp);
    if (e != cudaSuccess) return fail(e, "cudaGraphAddNode (while)");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e, "capture (PCG body)");
    const long long lb0 = c.launches;
    for (int par = 0; par < 2; ++par) {   // two PCG steps; FFT pass directions alternate as in op_solve_z
        if (fft) {
            k_cols<T><<<grid_for(c, pcol.n), kFftThreads, smem_c, c.stream>>>(pcol.view(), c.d_geom, c.d_const,
                                                                              c.d_state, P, pre, tw, half_c, par);
            k_pcg_inv<T><<<grid_for(c, prow.n), kFftThreads, smem, c.stream>>>(prow.view(), c.d_geom, c.d_state, P,
                                                                              tw, half, par, par ^ 1);
            c.launches += 2;
        }
        if (mg) mg_tail<T>(c, par, par, false);
        if (fft) {
            k_pcg_fwd<T, true><<<grid_for(c, prow.n), kFftThreads, smem, c.stream>>>(
                prow.view(), c.d_geom, c.d_const, c.d_state, P, tw, half, par, c.d_cg_pending, par);
            c.launches += 1;
        }
        if (mg) mg_fwd<T, true>(c, par, par, false);   // residual buffers alternate with the steps
    }
    const int per_body = (int)(c.launches - lb0) + 1;
    c.launches = lb0;   // counted on the device as the bodies run
    k_pcg_loop_cond<<<1, 1, 0, c.stream>>>(h, c.d_cg_pending, c.d_graph_body, bodies, c.d_graph_launches,
                                           per_body);
    e = cudaStreamEndCapture(c.stream, &body);
    if (e != cudaSuccess) return fail(e, "capture end (PCG body)");
    // 3. beta schedule after the loop
    e = cudaStreamBeginCaptureToGraph(c.stream, g, &cond, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e, "capture (iteration tail)");
    rc = op_next_beta<T>(c);
    e = cudaStreamEndCapture(c.stream, &g);
    c.stream = user;
    if (rc) {
        cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(e, "capture end (iteration tail)");
    e = cudaGraphInstantiate(&c.graph_exec, g, 0);
    if (e != cudaSuccess) return fail(e, "cudaGraphInstantiate");
    c.graph = g;
    c.graph_static_launches = c.launches - l0;
    c.launches = l0;
    return RECON_OK;
}

// One captured iteration on the graph stream, ordered after and before the
// work of the handle's stream.
template <typename T>
int graph_iterate_t(Ctx& c) {
    int rc;
    if (!c.graph_exec && (rc = graph_build_t<T>(c))) return rc;
    RECON_CUDA(cudaEventRecord(c.graph_ev[0], c.stream));
    RECON_CUDA(cudaStreamWaitEvent(c.graph_stream, c.graph_ev[0], 0));
    RECON_CUDA(cudaGraphLaunch(c.graph_exec, c.graph_stream));
    RECON_CUDA(cudaEventRecord(c.graph_ev[1], c.graph_stream));
    RECON_CUDA(cudaStreamWaitEvent(c.stream, c.graph_ev[1], 0));
    c.launches += c.graph_static_launches;
    return RECON_OK;
}

template <typename T>
int iterate_t(Ctx& c, bool stats) {
    int rc;
    if (c.domain == 1 && (rc = op_modeb_gram<T>(c))) return rc;
    if (c.domain == 2 && (rc = op_gn_terms(c))) return rc;
    if ((rc = op_thr_rhs<T>(c, stats))) return rc;
    if ((rc = c.domain != 0 ? op_solve_f_sino<T>(c) : op_solve_f<T>(c))) return rc;
    if ((rc = op_synth<T>(c))) return rc;
    const FftJobs rho = jobs1(RECON_F_RHS_RHO, 2, RECON_F_RHO, 2);
    if (!c.side_stream) {
        if ((rc = fft_solve<T>(c, rho))) return rc;
        if ((rc = op_solve_z<T>(c))) return rc;
        return op_next_beta<T>(c);
    }
    // The rho_e and Z^m updates of an iteration read only what the synthesis
    // wrote (Alg. 1, reading R1) and touch disjoint fields and spectra: the FFT
    // solve of rho_e (instruction-bound) runs on the side stream while the Z^m
    // PCG (bound by HBM) runs on the handle's stream.
    RECON_CUDA(cudaEventRecord(c.side_ev[0], c.stream));
    RECON_CUDA(cudaStreamWaitEvent(c.side_stream, c.side_ev[0], 0));
    const cudaStream_t main_stream = c.stream;
    c.stream = c.side_stream;
    rc = fft_solve<T>(c, rho);
    const cudaError_t e = cudaEventRecord(c.side_ev[1], c.side_stream);
    c.stream = main_stream;
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord (side stream)");
    rc = op_solve_z<T>(c);
    // the handle's stream waits for the side stream even when the PCG failed
    RECON_CUDA(cudaStreamWaitEvent(c.stream, c.side_ev[1], 0));
    if (rc) return rc;
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
int extract_t(Ctx& c, int s0, int s1, float* Z, float* rhoe, float* f1, float* f2) {
    // the tiles of slices s0 .. s1-1 (the list is in slice order; k_extract reads only the items)
    ItemList L = c.tiles.view();
    const int i0 = c.tiles.h_lo[s0], i1 = s1 < c.n ? c.tiles.h_lo[s1] : c.tiles.n;
    L.items += i0;
    L.n_items = i1 - i0;
    if (L.n_items <= 0) return RECON_OK;
    k_extract<T><<<grid_for(c, L.n_items), kStencilThreads, 0, c.stream>>>(L, c.d_geom, ptrs<T>(c), Z, rhoe, f1, f2,
                                                                           water_z(), z_exponent());
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

// Debug operator: q = [diag(a^2) + beta~ L] p for every slice, with p read
// from CG_P0 and q written to CG_Q, by the kernel that forms q in that
// slice's PCG (k_mg_pq on multigrid slices, k_pcg_inv on the others).  Each
// slice is put in mid-solve state with beta_cg = 1, y = 0 and a zero
// preconditioner spectrum, so both kernels form p = 0 + 1 * p_old exactly and
// then q = M p.  The PCG scalars of the handle are left in that state.
__global__ void k_zmv_state(int n, SliceState* S) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SliceState& st = S[s];
    st.cg_it = 1;
    st.cg_done = 0;
    set_betacg(st, 1.0);
}

__global__ void k_zmv_alpha(int n, SliceState* S) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    S[s].cg_done = 0;
    set_alpha(S[s], 1.0);
}

template <typename T>
int op_z_matvec(Ctx& c) {
    k_zmv_state<<<(c.n + 127) / 128, 128, 0, c.stream>>>(c.n, c.d_state);
    c.launches += 1;
    RECON_CUDA(cudaMemsetAsync(c.field[RECON_F_CG_Y], 0, c.elem * (size_t)c.pool_elems, c.stream));
    RECON_CUDA(cudaMemsetAsync(c.spec[0], 0, 2 * c.elem * (size_t)c.spec_elems, c.stream));
    const Ptrs<T> P = ptrs<T>(c);
    const bool mg = c.mg_max_lb > 0;
    if (mg) {
        if constexpr (std::is_same<T, float>::value) {
            // k_mgs_pq forms q for p.q (stored here); k_mgs_fwd forms it again for
            // r' = r - alpha q: with alpha = 1, r = 0 and z = 0 it writes -q to
            // CG_R and p to Z
            RECON_CUDA(cudaMemsetAsync(c.field[RECON_F_CG_R2], 0, c.elem * (size_t)c.pool_elems, c.stream));
            RECON_CUDA(cudaMemsetAsync(c.field[RECON_F_Z], 0, c.elem * (size_t)c.pool_elems, c.stream));
            const int rb = strip_rows(c, 0);
            strip_pass(
                c, 0,
                [&](const DevItemList& S) {
                    k_mgb_pq<true><<<grid_for(c, S.n), kStripThreads, band_smem_bytes<3>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_state, P, 0, rb);
                },
                [&](const DevItemList& S) {
                    k_mgs_pq<true><<<grid_for(c, S.n), kStripThreads, strip_smem_bytes<3>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_state, P, 0, rb);
                });
            k_zmv_alpha<<<(c.n + 127) / 128, 128, 0, c.stream>>>(c.n, c.d_state);
            c.launches += 1;
            strip_pass(
                c, 0,
                [&](const DevItemList& S) {
                    k_mgb_fwd<true><<<grid_for(c, S.n), kStripThreads, band_smem_bytes<4>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_mg_geom[1], c.d_const, c.d_state, P, 0, mg_r<T>(c, 1), mg_r<T>(c, 0),
                        field_t<T>(c, RECON_F_A2), static_cast<T*>(c.mg_pool[0]), c.d_cg_pending, rb, 0);
                },
                [&](const DevItemList& S) {
                    k_mgs_fwd<true><<<grid_for(c, S.n), kStripThreads, strip_smem_bytes<4>(), c.stream>>>(
                        S.view(), c.d_geom, c.d_mg_geom[1], c.d_const, c.d_state, P, 0, mg_r<T>(c, 1), mg_r<T>(c, 0),
                        field_t<T>(c, RECON_F_A2), static_cast<T*>(c.mg_pool[0]), c.d_cg_pending, rb, 0);
                });
        } else {
            const DevItemList& L0 = c.mg_tiles[0];
            k_mg_pq<T><<<grid_for(c, L0.n), kStencilThreads, 2 * sizeof(MgBufPq<T>), c.stream>>>(
                L0.view(), c.d_geom, c.d_state, P, 0);
            c.launches += 1;
        }
    }
    const DevItemList& prow = mg ? c.pcg_rows : c.rows;
    if (prow.n > 0) {
        k_pcg_inv<T><<<grid_for(c, prow.n), kFftThreads, fft_smem_bytes<T>(c), c.stream>>>(
            prow.view(), c.d_geom, c.d_state, P, static_cast<const cplx<T>*>(c.d_tw), fft_half_slots<T>(c), 0, 0);
        c.launches += 1;
    }
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

template <typename T>
int op_t(Ctx& c, int op) {
    switch (op) {
        case RECON_OP_INIT: return init_maps_t<T>(c);
        case RECON_OP_THRESH_RHS: {
            int rc;
            if (c.domain == 1 && (rc = op_modeb_gram<T>(c))) return rc;
            if (c.domain == 2 && (rc = op_gn_terms(c))) return rc;
            return op_thr_rhs<T>(c, false);
        }
        case RECON_OP_SOLVE_F: return c.domain != 0 ? op_solve_f_sino<T>(c) : op_solve_f<T>(c);
        case RECON_OP_SYNTH: return op_synth<T>(c);
        case RECON_OP_SOLVE_RHO: return fft_solve<T>(c, jobs1(RECON_F_RHS_RHO, 2, RECON_F_RHO, 2));
        case RECON_OP_SOLVE_Z: return op_solve_z<T>(c);
        case RECON_OP_NEXT_BETA: return op_next_beta<T>(c);
        case RECON_OP_Z_MATVEC: return op_z_matvec<T>(c);
        default: set_error("unknown operator"); return RECON_EINVAL;
    }
}

SliceConst slice_const(const recon_params& p, const Tables& t) {
    SliceConst k{};
    k.a00 = t.a[0][0]; k.a01 = t.a[0][1]; k.a10 = t.a[1][0]; k.a11 = t.a[1][1];
    k.b00 = t.b[0][0]; k.b01 = t.b[0][1]; k.b10 = t.b[1][0]; k.b11 = t.b[1][1];
    k.P1 = t.P[0]; k.P2 = t.P[1]; k.psi1 = t.psi[0]; k.psi2 = t.psi[1];
    k.r = t.r; k.c_f1 = t.c_f[0]; k.c_f2 = t.c_f[1]; k.c12 = t.c12; k.c_rho = t.c_rho; k.a_w = t.a_w;
    k.det = t.det; k.inv_S = 1.0 / t.S; k.zclip_hi = t.zclip_hi; k.rho_air = p.rho_air;
    k.lambda = p.lambda; k.beta0 = p.beta0; k.tau = p.tau;
    k.kappa = p.kappa > 0 ? p.kappa : (p.iters > 0 ? std::pow(p.beta_max / p.beta0, 1.0 / p.iters) : 1.0);
    k.cg_tol = p.cg_tol; k.iters = p.iters; k.order = p.order; k.cg_max = p.cg_max_iters;
    k.domain = p.domain;
    k.fa0 = t.a[0][0] * t.a[0][0] + t.a[0][1] * t.a[0][1];
    k.fa1 = t.a[1][0] * t.a[1][0] + t.a[1][1] * t.a[1][1];
    k.fcp0 = t.b[0][0] * t.b[0][0] + t.b[0][1] * t.b[0][1];
    k.fcp1 = t.b[1][0] * t.b[1][0] + t.b[1][1] * t.b[1][1];
    k.fcross = t.a[0][0] * t.a[1][0] + t.a[0][1] * t.a[1][1];
    k.inv_gamma = 0.0;   // set once the geometry's gamma is known
    finish_const(k);
    return k;
}

// Work-item lists of one slice (tiles, row-pair groups, column groups) and
// its FFT batching, appended to the three lists.
// Row pairs per row-FFT item and columns per column-FFT item of an nx x ny
// slice, sized so one item's transforms fill about `budget` complex slots.
int rows_per_item(int nx, int ny, int budget) {
    const int npairs = (ny + 1) / 2;
    int per = budget / nx - 1;   // k_pcg_inv transforms one more pair (the halo rows)
    if (per < 1) per = 1;
    return per > npairs ? npairs : per;
}

int cols_per_item(int nx, int ny, int budget) {
    int pc = budget / ny;
    if (pc > 16) pc = 16;
    if (pc < 1) pc = 1;
    return pc > nx / 2 + 1 ? nx / 2 + 1 : pc;
}

// Complex slots of one FFT buffer for an nx x ny slice.
int fft_item_slots(int nx, int ny, int budget) {
    const int r = (rows_per_item(nx, ny, budget) + 1) * padded_len(nx);
    const int q = cols_per_item(nx, ny, budget) * col_ld(ny);
    return r > q ? r : q;
}

void slice_items(Ctx& c, int s, std::vector<Item>& tiles, std::vector<Item>& rows, std::vector<Item>& cols) {
    SliceGeom& g = c.sg[s];
    g.inv_n = (float)(1.0 / ((double)g.nx * (double)g.ny));
    const int budget = c.precision == 1 ? FftBudget<float>::E : FftBudget<double>::E;
    const int th = c.precision == 1 ? kTileHFloat : kTileHDouble;
    for (int ty = 0; ty < g.ny; ty += th)
        for (int tx = 0; tx < g.nx; tx += kTileW) tiles.push_back(Item{s, tx, ty, 0});
    const int npairs = (g.ny + 1) / 2;
    const int per = rows_per_item(g.nx, g.ny, c.row_budget > 0 ? c.row_budget : budget);
    g.rows_per_item = per;
    for (int p0 = 0; p0 < npairs; p0 += per) rows.push_back(Item{s, p0, (npairs - p0 < per ? npairs - p0 : per), 0});
    const int pc = cols_per_item(g.nx, g.ny, budget);
    g.cols_per_item = pc;
    for (int c0 = 0; c0 < g.nh; c0 += pc) cols.push_back(Item{s, c0, (g.nh - c0 < pc ? g.nh - c0 : pc), 0});
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
    L.cap = L.n;
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

// Row and column items of the FFT-preconditioned PCG: those of c.rows and
// c.cols on the slices without multigrid levels; and the tiles of k_cg_init:
// those of c.tiles on the slices whose fine level has no band items
// (k_mgb_start starts the others).  Host vectors.
void pcg_split_host(Ctx& c) {
    const std::vector<int>& band = c.mg_strips.empty() ? std::vector<int>() : c.mg_strips[0].h_cnt;
    const std::tuple<const DevItemList*, DevItemList*, int> parts[3] = {
        {&c.rows, &c.pcg_rows, 0}, {&c.cols, &c.pcg_cols, 0}, {&c.tiles, &c.cg_tiles, 1}};
    for (const auto& pr : parts) {
        const DevItemList& A = *std::get<0>(pr);
        DevItemList& B = *std::get<1>(pr);
        const bool tiles = std::get<2>(pr) != 0;
        B.h_items.clear();
        B.h_lo.assign(c.n, 0);
        B.h_cnt.assign(c.n, 0);
        for (int s = 0; s < c.n; ++s) {
            B.h_lo[s] = (int)B.h_items.size();
            if (tiles ? (!band.empty() && band[s] > 0) : c.mg_lb[s] != 0) continue;
            for (int i = 0; i < A.h_cnt[s]; ++i) B.h_items.push_back(A.h_items[A.h_lo[s] + i]);
            B.h_cnt[s] = A.h_cnt[s];
        }
    }
}

// Tile levels below the own grid of an nx x ny slice before its block level
// (at most kMgBlockPx pixels); 0 when the slice takes the FFT preconditioner.
// Each halving needs even sides, and the block level must halve on to at
// most kMgCoarsePx pixels.
int mg_tile_levels(int nx, int ny, int precision) {
    // the FP32 fine-level strip kernels take whole 16-byte vectors per lane and
    // two lanes at least in a row's last strip
    if (precision == 1 && nx % 8) return 0;
    int lb = 0;
    while ((long long)nx * ny > kMgBlockPx) {
        if (nx % 2 || ny % 2) return 0;
        nx /= 2;
        ny /= 2;
        ++lb;
    }
    if (lb == 0) return 0;
    int bx[kMgMaxBlockLevels], by[kMgMaxBlockLevels];
    const int J = mg_block_levels(nx, ny, bx, by);
    return bx[J - 1] * by[J - 1] <= kMgCoarsePx ? lb : 0;
}

// Shared-memory limits of the pipelined multigrid kernels (two buffers each).
template <typename T>
int mg_set_smem() {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    RECON_CUDA(cudaFuncSetAttribute(k_mg_fwd<T, false>, A, (int)(2 * sizeof(MgBufFwd<T>))));
    RECON_CUDA(cudaFuncSetAttribute(k_mg_fwd<T, true>, A, (int)(2 * sizeof(MgBufFwd<T>))));
    RECON_CUDA(cudaFuncSetAttribute(k_mg_down<T>, A, (int)(2 * sizeof(MgBufHalo2<T>))));
    RECON_CUDA(cudaFuncSetAttribute(k_mg_up<T>, A, (int)(2 * sizeof(MgBufHalo2<T>))));
    RECON_CUDA(cudaFuncSetAttribute(k_mg_y<T>, A, (int)(2 * sizeof(MgBufHalo2<T>))));
    RECON_CUDA(cudaFuncSetAttribute(k_mg_pq<T>, A, (int)(2 * sizeof(MgBufPq<T>))));
    return RECON_OK;
}

// Levels, pools and item lists of the multigrid preconditioner, and the row
// and column items of the slices that keep the FFT preconditioner.
int fill_list(Ctx& c, DevItemList& L);
int pcg_split_lists(Ctx& c);

// Items of the threshold pass: band items (kThrRows rows per band) of the
// FP32 slices whose width is a multiple of 4 and at most kBandMaxW, and the
// tiles of c.tiles on the other slices.  Host vectors.
void thr_split_host(Ctx& c) {
    DevItemList& B = c.thr_band;
    DevItemList& T = c.thr_tiles;
    for (DevItemList* X : {&B, &T}) {
        X->h_items.clear();
        X->h_lo.assign(c.n, 0);
        X->h_cnt.assign(c.n, 0);
    }
    for (int s = 0; s < c.n; ++s) {
        B.h_lo[s] = (int)B.h_items.size();
        T.h_lo[s] = (int)T.h_items.size();
        const int nx = c.sg[s].nx, ny = c.sg[s].ny;
        if (c.tiles.h_cnt[s] > 0 && c.precision == 1 && nx % 4 == 0 && nx <= kBandMaxW) {
            const int bh = band_groups(nx) * kThrRows;
            for (int y0 = 0; y0 < ny; y0 += bh) B.h_items.push_back(Item{s, 0, y0, 0});
        } else {
            for (int i = 0; i < c.tiles.h_cnt[s]; ++i) T.h_items.push_back(c.tiles.h_items[c.tiles.h_lo[s] + i]);
        }
        B.h_cnt[s] = (int)B.h_items.size() - B.h_lo[s];
        T.h_cnt[s] = (int)T.h_items.size() - T.h_lo[s];
    }
}

// Multigrid level l of slice s runs on the strip kernels (FP32, width a
// multiple of 8) rather than the tile kernels.
bool mg_strip_level(const Ctx& c, int s, int l) {
    return c.precision == 1 && c.mg_lb[s] > l && ((c.sg[s].nx >> l) % 8) == 0;
}

// Items of the multigrid level l of every slice in `slots` (every slice when
// null): strips (128 columns, kStripWarps x strip_rows rows) where
// mg_strip_level holds, and tiles (for the tile kernels) on the other slices
// with that level.  Host lists only.
// Resident blocks of the coarse band kernels over the device's SMs.
int band_resident(Ctx& c) {
    if (c.band_res > 0) return c.band_res;
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_mgb_fwd<false>, kStripThreads, band_smem_bytes<4>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mgb_up<false>, kStripThreads, band_smem_bytes<3>()) !=
            cudaSuccess) {
        cudaGetLastError();
        a = b = 4;   // the kernels' launch bounds
    }
    const int m = a < b ? a : b;
    c.band_res = (m > 0 ? m : 1) * c.sm_count;
    return c.band_res;
}

// Rows a warp walks per band item on a coarse level l >= 1 for the band
// items of `slots` (every slice when null).  The coarse passes form no
// reductions and every row's values come out the same whichever item forms
// them, so the count is free; it stays even (the restriction pairs rows from
// a band's first row).  The walks are bound by the latency of their row
// steps, so the count taken is the even one in [8, 32] that minimises the
// waves of resident blocks the items need times the rows one walks (its rows
// plus about 6 rows of halo and start); 0 (the default) without band items.
int coarse_band_rows(Ctx& c, int l, const std::vector<int>* slots) {
    const long long res = band_resident(c);
    int best = 0;
    long long best_cost = 0;
    for (int rb = 8; rb <= 32; rb += 2) {
        long long items = 0;
        auto count = [&](int s) {
            const int nx = c.sg[s].nx >> l;
            if (c.mg_lb[s] > l && mg_strip_level(c, s, l) && nx <= kBandMaxW && c.prm[s].pcg_kernel != 3) {
                const int bh = band_groups(nx) * rb;
                items += ((c.sg[s].ny >> l) + bh - 1) / bh;
            }
        };
        if (!slots)
            for (int s = 0; s < c.n; ++s) count(s);
        else
            for (int s : *slots) count(s);
        if (items == 0) return 0;
        const long long cost = (items + res - 1) / res * (rb + 6);
        if (!best || cost <= best_cost) {   // ties: the longer walk (fewer items)
            best = rb;
            best_cost = cost;
        }
    }
    return best;
}

void level_items(Ctx& c, int l, const std::vector<int>* slots) {
    if (l >= 1) {
        if ((int)c.mg_level_rb.size() <= l) c.mg_level_rb.resize(l + 1, 0);
        c.mg_level_rb[l] = c.precision == 1 ? coarse_band_rows(c, l, slots) : 0;
    }
    DevItemList& B = c.mg_strips[l];
    DevItemList& W = c.mg_wide[l];
    DevItemList& T = c.mg_tiles_rest[l];
    for (DevItemList* X : {&B, &W, &T}) {
        X->h_items.clear();
        X->h_lo.assign(c.n, 0);
        X->h_cnt.assign(c.n, 0);
    }
    const int rb = strip_rows(c, l);
    const int th = c.precision == 1 ? kTileHFloat : kTileHDouble;
    auto add = [&](int s) {
        for (DevItemList* X : {&B, &W, &T}) X->h_lo[s] = (int)X->h_items.size();
        if (c.mg_lb[s] > l) {
            const int nx = c.sg[s].nx >> l, ny = c.sg[s].ny >> l;
            if (mg_strip_level(c, s, l) && nx <= kBandMaxW && c.prm[s].pcg_kernel != 3) {
                const int bh = band_groups(nx) * rb;
                for (int y0 = 0; y0 < ny; y0 += bh) B.h_items.push_back(Item{s, 0, y0, 0});
            } else if (mg_strip_level(c, s, l)) {
                const int bh = kStripWarps * rb;
                for (int y0 = 0; y0 < ny; y0 += bh)
                    for (int x0 = 0; x0 < nx; x0 += kStripW) W.h_items.push_back(Item{s, x0, y0, 0});
            } else {
                for (int ty = 0; ty < ny; ty += th)
                    for (int tx = 0; tx < nx; tx += kTileW) T.h_items.push_back(Item{s, tx, ty, 0});
            }
        }
        for (DevItemList* X : {&B, &W, &T}) X->h_cnt[s] = (int)X->h_items.size() - X->h_lo[s];
    };
    if (!slots)
        for (int s = 0; s < c.n; ++s) add(s);
    else
        for (int s : *slots) add(s);
}

// Tiles of the multigrid levels 0 .. mg_max_lb - 1 of the given slots (a
// slot's level l has tiles while mg_lb > l), uploaded.
int mg_lists_for(Ctx& c, const std::vector<int>& slots) {
    const int th = c.precision == 1 ? kTileHFloat : kTileHDouble;
    int rc;
    for (int l = 0; l < c.mg_max_lb; ++l) {
        DevItemList& T = c.mg_tiles[l];
        T.h_items.clear();
        T.h_lo.assign(c.n, 0);
        T.h_cnt.assign(c.n, 0);
        for (int s : slots) {
            T.h_lo[s] = (int)T.h_items.size();
            if (c.mg_lb[s] <= l) continue;
            const int nx = c.sg[s].nx >> l, ny = c.sg[s].ny >> l;
            for (int ty = 0; ty < ny; ty += th)
                for (int tx = 0; tx < nx; tx += kTileW) T.h_items.push_back(Item{s, tx, ty, 0});
            T.h_cnt[s] = (int)T.h_items.size() - T.h_lo[s];
        }
        if ((rc = fill_list(c, T))) return rc;
    }
    for (int l = 0; l < c.mg_max_lb; ++l) {
        level_items(c, l, &slots);
        if ((rc = fill_list(c, c.mg_strips[l])) || (rc = fill_list(c, c.mg_wide[l])) ||
            (rc = fill_list(c, c.mg_tiles_rest[l])))
            return rc;
    }
    return pcg_split_lists(c);
}

// Serving engine: every slot gets the multigrid levels of the capacity at
// fixed offsets (like its fields); a slot's levels are sized when a request
// is configured into it (mg_configure_slot).
int mg_setup_server(Ctx& c) {
    int rc;
    int L = 0;
    for (int nx = c.cap_nx, ny = c.cap_ny; (long long)nx * ny > kMgBlockPx && nx > 1 && ny > 1; nx /= 2, ny /= 2) ++L;
    if (L == 0) return RECON_OK;
    c.mg_max_lb = L;
    c.mg_sg.assign(L + 1, std::vector<SliceGeom>(c.n, SliceGeom{}));
    long long off = 0;
    for (int l = 1; l <= L; ++l)
        for (int s = 0; s < c.n; ++s) {
            SliceGeom& g = c.mg_sg[l][s];
            g.pitch = ((c.cap_nx >> l) + 31) / 32 * 32;
            g.off = off;
            g.lvl = l;
            off += (long long)(c.cap_ny >> l) * g.pitch;
        }
    for (int k = 0; k < 3; ++k) {
        if ((rc = alloc_dev(c, &c.mg_pool[k], c.elem * off))) return rc;
        RECON_CUDA(cudaMemset(c.mg_pool[k], 0, c.elem * off));
    }
    c.d_mg_geom.assign(L + 1, nullptr);
    c.d_mg_geom[0] = c.d_geom;
    for (int l = 1; l <= L; ++l) {
        if ((rc = alloc_dev(c, (void**)&c.d_mg_geom[l], sizeof(SliceGeom) * c.n))) return rc;
        RECON_CUDA(cudaMemcpy(c.d_mg_geom[l], c.mg_sg[l].data(), sizeof(SliceGeom) * c.n, cudaMemcpyHostToDevice));
    }
    const std::vector<SliceGeom> blk(c.n, SliceGeom{});
    if ((rc = alloc_dev(c, (void**)&c.d_mg_block, sizeof(SliceGeom) * c.n))) return rc;
    RECON_CUDA(cudaMemcpy(c.d_mg_block, blk.data(), sizeof(SliceGeom) * c.n, cudaMemcpyHostToDevice));
    // the largest block level any slot can have: at most kMgBlockPx pixels and its coarser grids
    int tot = 0;
    for (int px = kMgBlockPx; px >= 1; px /= 4) tot += px;
    c.mg_block_smem = (3 * tot + kMgBlockPx) * (int)c.elem;
    c.mg_inv_smem = kMgCoarseInvSmem + tot * (int)c.elem + (int)c.elem;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (c.precision == 1) {
        RECON_CUDA(cudaFuncSetAttribute(k_mg_block<float>, A, c.mg_block_smem));
        RECON_CUDA(cudaFuncSetAttribute(k_mg_coarse_inv<float>, A, c.mg_inv_smem));
    } else {
        RECON_CUDA(cudaFuncSetAttribute(k_mg_block<double>, A, c.mg_block_smem));
        RECON_CUDA(cudaFuncSetAttribute(k_mg_coarse_inv<double>, A, c.mg_inv_smem));
    }
    if ((rc = alloc_dev(c, &c.mg_qinv, c.elem * (size_t)kMgCoarsePx * kMgCoarsePx * c.n))) return rc;
    if ((rc = c.precision == 1 ? mg_set_smem<float>() : mg_set_smem<double>())) return rc;
    c.mg_tiles.assign(L, DevItemList{});
    for (int l = 0; l < L; ++l) {
        c.mg_tiles[l].h_lo.assign(c.n, 0);
        c.mg_tiles[l].h_cnt.assign(c.n, 0);
        if ((rc = upload_list(c, c.mg_tiles[l]))) return rc;
    }
    c.mg_strips.assign(L, DevItemList{});
    c.mg_wide.assign(L, DevItemList{});
    c.mg_tiles_rest.assign(L, DevItemList{});
    for (int l = 0; l < L; ++l) {
        const std::vector<int> none;
        level_items(c, l, &none);
        if ((rc = upload_list(c, c.mg_strips[l])) || (rc = upload_list(c, c.mg_wide[l])) ||
            (rc = upload_list(c, c.mg_tiles_rest[l])))
            return rc;
    }
    pcg_split_host(c);
    if ((rc = upload_list(c, c.pcg_rows)) || (rc = upload_list(c, c.pcg_cols)) || (rc = upload_list(c, c.cg_tiles)))
        return rc;
    return RECON_OK;
}

int mg_setup(Ctx& c) {
    int rc;
    c.mg_lb.assign(c.n, 0);
    c.mg_max_lb = 0;
    if (c.server_mode) return mg_setup_server(c);
    if (c.prm[0].pcg_kernel == 2) return RECON_OK;
    for (int s = 0; s < c.n; ++s) {
        c.mg_lb[s] = mg_tile_levels(c.sg[s].nx, c.sg[s].ny, c.precision);
        c.mg_max_lb = c.mg_lb[s] > c.mg_max_lb ? c.mg_lb[s] : c.mg_max_lb;
    }
    if (c.mg_max_lb == 0) return RECON_OK;
    const int L = c.mg_max_lb;
    // grids of levels 1 .. L (one pool per quantity, every level of every slice)
    c.mg_sg.assign(L + 1, std::vector<SliceGeom>(c.n, SliceGeom{}));
    long long off = 0;
    for (int l = 1; l <= L; ++l)
        for (int s = 0; s < c.n; ++s) {
            if (c.mg_lb[s] < l) continue;
            SliceGeom& g = c.mg_sg[l][s];
            g.nx = c.sg[s].nx >> l;
            g.ny = c.sg[s].ny >> l;
            g.pitch = (g.nx + 31) / 32 * 32;
            g.off = off;
            g.lvl = l;
            off += (long long)g.ny * g.pitch;
        }
    for (int k = 0; k < 3; ++k) {
        if ((rc = alloc_dev(c, &c.mg_pool[k], c.elem * off))) return rc;
        RECON_CUDA(cudaMemset(c.mg_pool[k], 0, c.elem * off));
    }
    c.d_mg_geom.assign(L + 1, nullptr);
    c.d_mg_geom[0] = c.d_geom;
    for (int l = 1; l <= L; ++l) {
        if ((rc = alloc_dev(c, (void**)&c.d_mg_geom[l], sizeof(SliceGeom) * c.n))) return rc;
        RECON_CUDA(cudaMemcpy(c.d_mg_geom[l], c.mg_sg[l].data(), sizeof(SliceGeom) * c.n, cudaMemcpyHostToDevice));
    }
    std::vector<SliceGeom> blk(c.n, SliceGeom{});
    int smem = 0;
    for (int s = 0; s < c.n; ++s) {
        if (!c.mg_lb[s]) continue;
        blk[s] = c.mg_sg[c.mg_lb[s]][s];
        int bx[kMgMaxBlockLevels], by[kMgMaxBlockLevels];
        const int J = mg_block_levels(blk[s].nx, blk[s].ny, bx, by);
        int tot = 0;
        for (int j = 0; j < J; ++j) tot += bx[j] * by[j];
        const int bytes = (3 * tot + bx[0] * by[0]) * (int)c.elem;
        smem = bytes > smem ? bytes : smem;
    }
    if ((rc = alloc_dev(c, (void**)&c.d_mg_block, sizeof(SliceGeom) * c.n))) return rc;
    RECON_CUDA(cudaMemcpy(c.d_mg_block, blk.data(), sizeof(SliceGeom) * c.n, cudaMemcpyHostToDevice));
    c.mg_block_smem = smem;
    // k_mg_coarse_inv: the dense operator and a^2 of every level (within a third of k_mg_block's share)
    c.mg_inv_smem = kMgCoarseInvSmem + smem / 3 + (int)c.elem;
    if (c.precision == 1) {
        RECON_CUDA(cudaFuncSetAttribute(k_mg_block<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        RECON_CUDA(cudaFuncSetAttribute(k_mg_coarse_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        c.mg_inv_smem));
    } else {
        RECON_CUDA(cudaFuncSetAttribute(k_mg_block<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        RECON_CUDA(cudaFuncSetAttribute(k_mg_coarse_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        c.mg_inv_smem));
    }
    if ((rc = alloc_dev(c, &c.mg_qinv, c.elem * (size_t)kMgCoarsePx * kMgCoarsePx * c.n))) return rc;
    if ((rc = c.precision == 1 ? mg_set_smem<float>() : mg_set_smem<double>())) return rc;
    // tiles of levels 0 .. L-1
    const int th = c.precision == 1 ? kTileHFloat : kTileHDouble;
    c.mg_tiles.assign(L, DevItemList{});
    for (int l = 0; l < L; ++l) {
        DevItemList& T = c.mg_tiles[l];
        T.h_lo.assign(c.n, 0);
        T.h_cnt.assign(c.n, 0);
        for (int s = 0; s < c.n; ++s) {
            T.h_lo[s] = (int)T.h_items.size();
            if (c.mg_lb[s] <= l) continue;
            const int nx = c.sg[s].nx >> l, ny = c.sg[s].ny >> l;
            for (int ty = 0; ty < ny; ty += th)
                for (int tx = 0; tx < nx; tx += kTileW) T.h_items.push_back(Item{s, tx, ty, 0});
            T.h_cnt[s] = (int)T.h_items.size() - T.h_lo[s];
        }
        if ((rc = upload_list(c, T))) return rc;
    }
    c.mg_strips.assign(L, DevItemList{});
    c.mg_wide.assign(L, DevItemList{});
    c.mg_tiles_rest.assign(L, DevItemList{});
    for (int l = 0; l < L; ++l) {
        level_items(c, l, nullptr);
        if ((rc = upload_list(c, c.mg_strips[l])) || (rc = upload_list(c, c.mg_wide[l])) ||
            (rc = upload_list(c, c.mg_tiles_rest[l])))
            return rc;
    }
    // row and column items of the PCG on the slices that keep the FFT preconditioner
    pcg_split_host(c);
    if ((rc = upload_list(c, c.pcg_rows)) || (rc = upload_list(c, c.pcg_cols)) || (rc = upload_list(c, c.cg_tiles)))
        return rc;
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
    for (DevItemList* L : {&c.tiles, &c.rows, &c.cols}) {
        L->h_lo.assign(c.n, 0);
        L->h_cnt.assign(c.n, 0);
        L->h_items.clear();
    }
    for (int s = 0; s < c.n; ++s) {
        SliceGeom& g = c.sg[s];
        const size_t t0 = c.tiles.h_items.size(), r0 = c.rows.h_items.size(), c0 = c.cols.h_items.size();
        slice_items(c, s, c.tiles.h_items, c.rows.h_items, c.cols.h_items);
        c.tiles.h_lo[s] = (int)t0;
        c.tiles.h_cnt[s] = (int)(c.tiles.h_items.size() - t0);
        c.rows.h_lo[s] = (int)r0;
        c.rows.h_cnt[s] = (int)(c.rows.h_items.size() - r0);
        c.cols.h_lo[s] = (int)c0;
        c.cols.h_cnt[s] = (int)(c.cols.h_items.size() - c0);
        g.plan_x = fft_plan_code(g.nx);
        g.plan_y = fft_plan_code(g.ny);
    }
    // twiddle tables exp(-2 pi i t / N), one per distinct N
    {
        std::vector<double> tw, sym;
        std::vector<std::pair<int, std::pair<long long, long long>>> have;
        auto table = [&](int n) -> std::pair<long long, long long> {
            for (auto& h : have)
                if (h.first == n) return h.second;
            const long long off = (long long)tw.size() / 2, soff = (long long)sym.size();
            for (int t = 0; t < n; ++t) {
                const double a = 2.0 * M_PI * (double)t / (double)n;
                tw.push_back(std::cos(a));
                tw.push_back(-std::sin(a));
                const double sn = std::sin(M_PI * (double)t / (double)n);
                sym.push_back(4.0 * sn * sn);
            }
            // compile-time transforms: stage-major table after the N entries
            // (layout of P2Plan in fft.cuh)
            if ((n >= 64 && n <= 1024 && (n & (n - 1)) == 0) || n == 320 || n == 384 || n == 448) {
                std::vector<int> radices;
                int m2 = n, l = 0;
                while (m2 % 2 == 0) { m2 /= 2; ++l; }
                for (int i = 0; i < l / 3; ++i) radices.push_back(8);
                if (l % 3) radices.push_back(l % 3 == 2 ? 4 : 2);
                for (int f : {3, 5, 7})
                    while (m2 % f == 0) {
                        m2 /= f;
                        radices.push_back(f);
                    }
                int ns = 1;
                for (size_t st = 0; st < radices.size(); ++st) {
                    const int R = radices[st];
                    if (st > 0) {
                        std::vector<int> pw;
                        if (R % 2 == 1)
                            for (int q = 1; q < R; ++q) pw.push_back(q);
                        else
                            for (int q : {1, 2, 4})
                                if (q < R) pw.push_back(q);
                        for (int q : pw)
                            for (int k = 0; k < ns; ++k) {
                                const double a = 2.0 * M_PI * (double)(q * k) / (double)(ns * R);
                                tw.push_back(std::cos(a));
                                tw.push_back(-std::sin(a));
                            }
                    }
                    ns *= R;
                }
            }
            have.push_back({n, {off, soff}});
            return {off, soff};
        };
        if (c.server_mode) {
            const int top = c.cap_nx > c.cap_ny ? c.cap_nx : c.cap_ny;
            for (int n = 1; n <= top; ++n) {
                int m = n;
                for (int f : {2, 3, 5, 7})
                    while (m % f == 0) m /= f;
                if (m == 1) table(n);
            }
        }
        for (SliceGeom& g : c.sg) {
            const auto tx = table(g.nx), ty = table(g.ny);
            g.twx = tx.first;
            g.symx = tx.second;
            g.twy = ty.first;
            g.symy = ty.second;
        }
        c.tw_index = have;
        if ((rc = alloc_dev(c, &c.d_tw, c.elem * tw.size()))) return rc;
        if ((rc = alloc_dev(c, &c.d_sym, c.elem * sym.size()))) return rc;
        if (c.precision == 1) {
            std::vector<float> f(tw.begin(), tw.end()), fs(sym.begin(), sym.end());
            RECON_CUDA(cudaMemcpy(c.d_tw, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
            RECON_CUDA(cudaMemcpy(c.d_sym, fs.data(), sizeof(float) * fs.size(), cudaMemcpyHostToDevice));
        } else {
            RECON_CUDA(cudaMemcpy(c.d_tw, tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice));
            RECON_CUDA(cudaMemcpy(c.d_sym, sym.data(), sizeof(double) * sym.size(), cudaMemcpyHostToDevice));
        }
    }
    if ((rc = upload_list(c, c.tiles)) || (rc = upload_list(c, c.rows)) || (rc = upload_list(c, c.cols))) return rc;
    thr_split_host(c);
    if ((rc = upload_list(c, c.thr_band)) || (rc = upload_list(c, c.thr_tiles))) return rc;
    if (c.precision == 1) {
        RECON_CUDA(cudaFuncSetAttribute(k_thr_band<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        band_smem_bytes<6>()));
        RECON_CUDA(cudaFuncSetAttribute(k_thr_band<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        band_smem_bytes<8>()));
    }
    if (c.server_mode) {
        c.tmp_tiles.h_items = c.tiles.h_items;
        c.tmp_tiles.h_lo = c.tiles.h_lo;
        c.tmp_tiles.h_cnt = c.tiles.h_cnt;
        if ((rc = upload_list(c, c.tmp_tiles))) return rc;
    }
    // constants
    std::vector<SliceConst>& hc = c.hconst;
    hc.assign(c.n, SliceConst{});
    c.tab.resize(c.n);
    for (int s = 0; s < c.n; ++s) {
        c.tab[s] = make_tables(c.prm[s]);
        hc[s] = slice_const(c.prm[s], c.tab[s]);
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
    if ((rc = alloc_dev(c, (void**)&c.d_cg_pending, 2 * sizeof(int)))) return rc;
    if ((rc = alloc_dev(c, (void**)&c.d_acct, sizeof(unsigned long long) * KF_COUNT))) return rc;
    RECON_CUDA(cudaMemset(c.d_acct, 0, sizeof(unsigned long long) * KF_COUNT));
    RECON_CUDA(cudaMallocHost((void**)&c.h_cg_pending, 2 * sizeof(int)));
    RECON_CUDA(cudaStreamCreateWithFlags(&c.side_stream, cudaStreamNonBlocking));
    RECON_CUDA(cudaEventCreateWithFlags(&c.side_ev[0], cudaEventDisableTiming));
    RECON_CUDA(cudaEventCreateWithFlags(&c.side_ev[1], cudaEventDisableTiming));
    RECON_CUDA(cudaMemcpy(c.d_geom, c.sg.data(), sizeof(SliceGeom) * c.n, cudaMemcpyHostToDevice));
    if ((rc = mg_setup(c))) return rc;
    if (c.precision == 1)
        RECON_CUDA(cudaFuncSetAttribute(k_cg_init<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(2 * sizeof(CgInitBuf<float>))));
    else
        RECON_CUDA(cudaFuncSetAttribute(k_cg_init<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(2 * sizeof(CgInitBuf<double>))));
    if (c.precision == 1) return set_fft_smem<float>(c);
    return set_fft_smem<double>(c);
}

int solver_load_images(Ctx& c, const float* lo, const float* hi, int /*on_device*/) {
    return c.precision == 1 ? load_t<float>(c, lo, hi) : load_t<double>(c, lo, hi);
}

int solver_init_maps(Ctx& c) { return c.precision == 1 ? init_maps_t<float>(c) : init_maps_t<double>(c); }

int solver_setup_sino(Ctx& c) {
    const recon_geometry& g = c.geo[0];
    const long long nr = (long long)g.n_views * g.n_bins;
    int rc;
    if ((rc = alloc_dev(c, (void**)&c.d_sino_tmp, sizeof(float) * nr * c.n))) return rc;
    // gamma = ||A 1||^2 / (nx ny)
    float* ones = nullptr;
    RECON_CUDA(cudaMalloc((void**)&ones, sizeof(float) * g.nx * g.ny));
    std::vector<float> h(std::max<long long>(nr, (long long)g.nx * g.ny), 1.f);
    cudaError_t e = cudaMemcpy(ones, h.data(), sizeof(float) * g.nx * g.ny, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        rc = ct_project_pitched(g, 1, ones, g.nx, (long long)g.nx * g.ny, c.d_sino_tmp, c.stream, &c.launches);
        if (!rc) e = cudaStreamSynchronize(c.stream);
        if (!rc && e == cudaSuccess) e = cudaMemcpy(h.data(), c.d_sino_tmp, sizeof(float) * nr, cudaMemcpyDeviceToHost);
    }
    cudaFree(ones);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "gamma of the projector");
    double s2 = 0.0;
    for (long long i = 0; i < nr; ++i) s2 += (double)h[i] * (double)h[i];
    c.gamma = s2 / ((double)g.nx * (double)g.ny);
    if (!(c.gamma > 0.0)) {
        set_error("domain 1: the projector misses the image (gamma = 0)");
        return RECON_EINVAL;
    }
    const int domain = c.prm[0].domain;
    for (int s = 0; s < c.n; ++s) {
        c.hconst[s].inv_gamma = 1.0 / c.gamma;
        c.hconst[s].gn = domain == 2;
        finish_const(c.hconst[s]);
    }
    RECON_CUDA(cudaMemcpy(c.d_const, c.hconst.data(), sizeof(SliceConst) * c.n, cudaMemcpyHostToDevice));
    if (domain == 2) {
        // per-ray arrays, and the spectra of both arms with the basis values per bin
        if ((rc = alloc_dev(c, (void**)&c.d_gn, sizeof(float) * kGnArrays * nr * c.n))) return rc;
        const recon_params& p = c.prm[0];
        std::vector<float> tab;
        const recon_spectrum* arms[2] = {&p.low, &p.high};
        for (int a = 0; a < 2; ++a) {
            std::vector<double> E, w;
            spectrum_bins(*arms[a], E, w);
            c.spec_nb[a] = (int)E.size();
            for (size_t b = 0; b < E.size(); ++b) {
                tab.push_back((float)w[b]);
                tab.push_back((float)mu_norm(p.basis_z[0], p.basis_rhoe[0], E[b]));
                tab.push_back((float)mu_norm(p.basis_z[1], p.basis_rhoe[1], E[b]));
            }
        }
        if ((rc = alloc_dev(c, (void**)&c.d_spec, sizeof(float) * tab.size()))) return rc;
        RECON_CUDA(cudaMemcpy(c.d_spec, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
    }
    c.domain = domain;
    return RECON_OK;
}

int solver_modeb_data(Ctx& c) {
    // t_k = A^T ((a_k0 s_L + a_k1 s_H) / (S gamma)) into MUL (k = 0) and MUH (k = 1);
    // the initialisation has already used the FBP images held there
    const recon_geometry& g = c.geo[0];
    const long long nr = (long long)g.n_views * g.n_bins;
    const long long pitch = c.sg[0].pitch, stride = (long long)c.sg[0].ny * pitch;
    int rc;
    for (int k = 0; k < 2; ++k) {
        for (int s = 0; s < c.n; ++s) {
            const SliceConst& q = c.hconst[s];
            const double sc = q.inv_S * q.inv_gamma;
            const float wL = (float)((k ? q.a10 : q.a00) * sc), wH = (float)((k ? q.a11 : q.a01) * sc);
            k_sino_combine<<<(unsigned)((nr + 255) / 256), 256, 0, c.stream>>>(
                nr, c.d_sino[0] + c.sino_off[s], c.d_sino[1] + c.sino_off[s], wL, wH, c.d_sino_tmp + nr * s);
            c.launches += 1;
        }
        RECON_CUDA(cudaGetLastError());
        float* out = field_base<float>(c, k ? RECON_F_MUH : RECON_F_MUL);
        RECON_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * stride * c.n, c.stream));
        if ((rc = ct_backproject_add(g, c.n, c.d_sino_tmp, out, pitch, stride, c.stream, &c.launches))) return rc;
    }
    return RECON_OK;
}

// Time `reps` passes of one stencil kernel (k_cg_init) and one FFT solve
// (CG_R -> CG_Y, the rho_e divide) on fields the solve state does not use
// before the next iteration; returns the time in ms.
template <typename T>
int tune_time(Ctx& c, int reps, float* ms) {
    const Ptrs<T> P = ptrs<T>(c);
    cudaEvent_t a, b;
    RECON_CUDA(cudaEventCreate(&a));
    RECON_CUDA(cudaEventCreate(&b));
    int rc = RECON_OK;
    for (int r = -1; r < reps && !rc; ++r) {   // r = -1: warm-up
        if (r == 0) cudaEventRecord(a, c.stream);
        k_cg_init<T><<<grid_for(c, c.tiles.n), kStencilThreads, 2 * sizeof(CgInitBuf<T>), c.stream>>>(c.tiles.view(), c.d_geom, c.d_const,
                                                                              c.d_state, P, c.d_cg_pending);
        c.launches += 1;
        rc = fft_solve<T>(c, jobs1(RECON_F_CG_R, 0, RECON_F_CG_Y, 2));
    }
    cudaEventRecord(b, c.stream);
    cudaError_t e = cudaEventSynchronize(b);
    if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    return e == cudaSuccess ? RECON_OK : cuda_fail(e, "autotune timing");
}

void solver_free_graph(Ctx& c) {
    if (c.graph_exec) cudaGraphExecDestroy(c.graph_exec);
    if (c.graph) cudaGraphDestroy(c.graph);
    c.graph_exec = nullptr;
    c.graph = nullptr;
}

int solver_set_graph(Ctx& c, bool on) {
    if (on && (c.domain != 0 || c.server_mode)) {
        set_error("graph capture needs domain 0 and a solve handle");
        return RECON_EINVAL;
    }
    solver_free_graph(c);
    if (on && !c.graph_stream) {
        RECON_CUDA(cudaStreamCreateWithFlags(&c.graph_stream, cudaStreamNonBlocking));
        RECON_CUDA(cudaEventCreateWithFlags(&c.graph_ev[0], cudaEventDisableTiming));
        RECON_CUDA(cudaEventCreateWithFlags(&c.graph_ev[1], cudaEventDisableTiming));
        int rc;
        if ((rc = alloc_dev(c, (void**)&c.d_graph_body, sizeof(int)))) return rc;
        if ((rc = alloc_dev(c, (void**)&c.d_graph_launches, sizeof(unsigned long long)))) return rc;
        RECON_CUDA(cudaMemset(c.d_graph_launches, 0, sizeof(unsigned long long)));
    }
    c.graph_on = on;
    return RECON_OK;
}

long long solver_graph_loop_launches(Ctx& c) {
    if (!c.d_graph_launches) return 0;
    unsigned long long v = 0;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess || cudaStreamSynchronize(c.graph_stream) != cudaSuccess ||
        cudaMemcpy(&v, c.d_graph_launches, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return 0;
    return (long long)v;
}

namespace {
// Copy host item vectors into a device list allocated at capacity.
int fill_list(Ctx& c, DevItemList& L) {
    L.n = (int)L.h_items.size();
    if (L.n > L.cap) {   // more items than at setup (smaller row items): larger arrays
        int rc;
        if ((rc = alloc_dev(c, (void**)&L.items, sizeof(Item) * L.n))) return rc;
        if ((rc = alloc_dev(c, (void**)&L.partials, sizeof(double) * kMaxPartials * L.n))) return rc;
        L.cap = L.n;
    }
    if (L.n)
        RECON_CUDA(cudaMemcpyAsync(L.items, L.h_items.data(), sizeof(Item) * L.h_items.size(), cudaMemcpyHostToDevice,
                                   c.stream));
    RECON_CUDA(cudaMemcpyAsync(L.lo, L.h_lo.data(), sizeof(int) * c.n, cudaMemcpyHostToDevice, c.stream));
    RECON_CUDA(cudaMemcpyAsync(L.cnt, L.h_cnt.data(), sizeof(int) * c.n, cudaMemcpyHostToDevice, c.stream));
    RECON_CUDA(cudaStreamSynchronize(c.stream));   // host vectors may change right after
    return RECON_OK;
}

// The FFT-preconditioned PCG's row and column lists after c.rows and c.cols
// were rebuilt (no-op without multigrid slices: the PCG then uses c.rows and
// c.cols themselves).
int pcg_split_lists(Ctx& c) {
    if (c.mg_max_lb == 0) return RECON_OK;
    pcg_split_host(c);
    int rc;
    if ((rc = fill_list(c, c.pcg_rows)) || (rc = fill_list(c, c.pcg_cols)) || (rc = fill_list(c, c.cg_tiles)))
        return rc;
    return RECON_OK;
}

void lists_for(Ctx& c, const std::vector<int>& slots, DevItemList* tiles, DevItemList* rows, DevItemList* cols) {
    std::vector<Item> dr, dc;
    for (DevItemList* L : {tiles, rows, cols}) {
        if (!L) continue;
        L->h_items.clear();
        L->h_lo.assign(c.n, 0);
        L->h_cnt.assign(c.n, 0);
    }
    for (int s : slots) {
        const size_t t0 = tiles->h_items.size();
        const size_t r0 = rows ? rows->h_items.size() : 0, c0 = cols ? cols->h_items.size() : 0;
        slice_items(c, s, tiles->h_items, rows ? rows->h_items : dr, cols ? cols->h_items : dc);
        tiles->h_lo[s] = (int)t0;
        tiles->h_cnt[s] = (int)(tiles->h_items.size() - t0);
        if (rows) {
            rows->h_lo[s] = (int)r0;
            rows->h_cnt[s] = (int)(rows->h_items.size() - r0);
        }
        if (cols) {
            cols->h_lo[s] = (int)c0;
            cols->h_cnt[s] = (int)(cols->h_items.size() - c0);
        }
    }
}
}  // namespace

// Candidates: grid = {16, 32, 64} x SMs (the arithmetic is the same for all;
// items and their partial sums do not change), and with autotune = 2 (FP32)
// row items of {2048, 3072, 4096} complex slots, which regroups the per-item
// partial sums of the PCG reductions (last-bit differences).  Best of three
// timed passes each; the choice holds for the handle.
int solver_autotune(Ctx& c) {
    if (c.autotune == 0 || c.server_mode) return RECON_OK;
    std::vector<int> all(c.n);
    for (int s = 0; s < c.n; ++s) all[s] = s;
    std::vector<int> budgets = {c.row_budget};
    if (c.autotune == 2 && c.precision == 1) budgets = {2048, 3072, 4096};
    float best = 1e30f;
    int best_m = c.grid_mult, best_b = c.row_budget;
    int rc;
    for (int b : budgets) {
        c.row_budget = b;
        lists_for(c, all, &c.tiles, &c.rows, &c.cols);
        if ((rc = fill_list(c, c.tiles)) || (rc = fill_list(c, c.rows)) || (rc = fill_list(c, c.cols))) return rc;
        thr_split_host(c);
        if ((rc = fill_list(c, c.thr_band)) || (rc = fill_list(c, c.thr_tiles))) return rc;
        if ((rc = pcg_split_lists(c))) return rc;
        if ((rc = c.precision == 1 ? set_fft_smem<float>(c) : set_fft_smem<double>(c))) return rc;
        for (int m : {16, 32, 64}) {
            c.grid_mult = m;
            float ms = 0.f;
            if ((rc = c.precision == 1 ? tune_time<float>(c, 3, &ms) : tune_time<double>(c, 3, &ms))) return rc;
            if (ms < best) {
                best = ms;
                best_m = m;
                best_b = b;
            }
        }
    }
    c.grid_mult = best_m;
    c.row_budget = best_b;
    lists_for(c, all, &c.tiles, &c.rows, &c.cols);
    if ((rc = fill_list(c, c.tiles)) || (rc = fill_list(c, c.rows)) || (rc = fill_list(c, c.cols))) return rc;
    thr_split_host(c);
    if ((rc = fill_list(c, c.thr_band)) || (rc = fill_list(c, c.thr_tiles))) return rc;
    if ((rc = pcg_split_lists(c))) return rc;
    if ((rc = c.precision == 1 ? set_fft_smem<float>(c) : set_fft_smem<double>(c))) return rc;
    c.tuned = true;
    solver_free_graph(c);   // a captured graph holds the old launch shapes
    return RECON_OK;
}

int solver_iterate(Ctx& c, bool stats) {
    if (c.graph_on && !stats && c.prof_mask == 0)
        return c.precision == 1 ? graph_iterate_t<float>(c) : graph_iterate_t<double>(c);
    return c.precision == 1 ? iterate_t<float>(c, stats) : iterate_t<double>(c, stats);
}

int solver_op(Ctx& c, int op) { return c.precision == 1 ? op_t<float>(c, op) : op_t<double>(c, op); }

int solver_extract(Ctx& c, float* Z, float* rhoe, float* f1, float* f2, int /*on_device*/) {
    return solver_extract_range(c, 0, c.n, Z, rhoe, f1, f2);
}

int solver_extract_range(Ctx& c, int s0, int s1, float* Z, float* rhoe, float* f1, float* f2) {
    return c.precision == 1 ? extract_t<float>(c, s0, s1, Z, rhoe, f1, f2)
                            : extract_t<double>(c, s0, s1, Z, rhoe, f1, f2);
}

int solver_direct(Ctx& c, const float* lo, const float* hi, float* Z, float* rhoe) {
    const int grid = grid_for(c, c.tiles.n);
    if (c.precision == 1)
        k_direct<float><<<grid, kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, c.d_const, ptrs<float>(c),
                                                                lo, hi, Z, rhoe, water_z(), z_exponent());
    else
        k_direct<double><<<grid, kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, c.d_const,
                                                                 ptrs<double>(c), lo, hi, Z, rhoe, water_z(),
                                                                 z_exponent());
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

int solver_mono(Ctx& c, int n_e, const double* kev, float* out) {
    if (n_e < 1 || n_e > kMonoMax) {
        set_error("recon_mono: 1 to 16 energies per call");
        return RECON_EINVAL;
    }
    MonoCoef mc{};
    mc.n = n_e;
    const recon_params& p = c.prm[0];
    for (const recon_params& q : c.prm)
        if (q.basis_z[0] != p.basis_z[0] || q.basis_z[1] != p.basis_z[1] || q.basis_rhoe[0] != p.basis_rhoe[0] ||
            q.basis_rhoe[1] != p.basis_rhoe[1]) {
            set_error("recon_mono: the slices of the handle have different basis materials");
            return RECON_EINVAL;
        }
    for (int k = 0; k < n_e; ++k) {
        if (!(kev[k] > 0)) {
            set_error("recon_mono: energies must be positive (keV)");
            return RECON_EINVAL;
        }
        // every slice of a handle shares the basis materials (checked at init)
        for (int j = 0; j < 2; ++j) mc.c[k][j] = scale_per_mm() * mu_norm(p.basis_z[j], p.basis_rhoe[j], kev[k]);
    }
    const int grid = grid_for(c, c.tiles.n);
    if (c.precision == 1)
        k_mono<float><<<grid, kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, ptrs<float>(c), mc, out,
                                                              c.ext_elems);
    else
        k_mono<double><<<grid, kStencilThreads, 0, c.stream>>>(c.tiles.view(), c.d_geom, ptrs<double>(c), mc, out,
                                                               c.ext_elems);
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

__global__ void k_reset_slots(const int* slots, int n, const SliceConst* C, SliceState* S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = slots[i];
    const SliceConst& c = C[s];
    SliceState st = {};
    set_beta(st, c.beta0, c);
    st.active = c.iters > 0;
    st.cg_done = 1;
    S[s] = st;
}



int solver_configure_slot(Ctx& c, int s, const recon_geometry& geo, const recon_params& p) {
    if (!c.server_mode || s < 0 || s >= c.n) return RECON_EINVAL;
    if (geo.nx > c.cap_nx || geo.ny > c.cap_ny || p.precision != c.precision) {
        set_error("request exceeds the slot capacity or precision of the server");
        return RECON_EINVAL;
    }
    c.geo[s] = geo;
    c.prm[s] = p;
    SliceGeom& g = c.sg[s];
    g.nx = geo.nx;
    g.ny = geo.ny;
    g.nh = g.nx / 2 + 1;
    g.plan_x = fft_plan_code(g.nx);
    g.plan_y = fft_plan_code(g.ny);
    for (auto& h : c.tw_index) {
        if (h.first == g.nx) {
            g.twx = h.second.first;
            g.symx = h.second.second;
        }
        if (h.first == g.ny) {
            g.twy = h.second.first;
            g.symy = h.second.second;
        }
    }
    std::vector<Item> a, b, d;
    slice_items(c, s, a, b, d);   // sets rows_per_item / cols_per_item
    c.tab[s] = make_tables(p);
    c.hconst[s] = slice_const(p, c.tab[s]);
    if (c.mg_max_lb > 0) {
        // the request's multigrid levels inside the slot's capacity regions
        const int lb = p.pcg_kernel == 2 ? 0 : mg_tile_levels(geo.nx, geo.ny, c.precision);
        c.mg_lb[s] = lb;
        for (int l = 1; l <= c.mg_max_lb; ++l) {
            SliceGeom& gl = c.mg_sg[l][s];
            gl.nx = l <= lb ? geo.nx >> l : 0;
            gl.ny = l <= lb ? geo.ny >> l : 0;
            RECON_CUDA(cudaMemcpyAsync(c.d_mg_geom[l] + s, &gl, sizeof(SliceGeom), cudaMemcpyHostToDevice, c.stream));
        }
        const SliceGeom blk = lb ? c.mg_sg[lb][s] : SliceGeom{};
        RECON_CUDA(cudaMemcpyAsync(c.d_mg_block + s, &blk, sizeof(SliceGeom), cudaMemcpyHostToDevice, c.stream));
    }
    RECON_CUDA(cudaMemcpyAsync(c.d_geom + s, &c.sg[s], sizeof(SliceGeom), cudaMemcpyHostToDevice, c.stream));
    RECON_CUDA(cudaMemcpyAsync(c.d_const + s, &c.hconst[s], sizeof(SliceConst), cudaMemcpyHostToDevice, c.stream));
    RECON_CUDA(cudaStreamSynchronize(c.stream));
    return RECON_OK;
}

int solver_rebuild_lists(Ctx& c, const std::vector<int>& active) {
    lists_for(c, active, &c.tiles, &c.rows, &c.cols);
    int rc;
    if ((rc = fill_list(c, c.tiles)) || (rc = fill_list(c, c.rows)) || (rc = fill_list(c, c.cols))) return rc;
    thr_split_host(c);
    if ((rc = fill_list(c, c.thr_band)) || (rc = fill_list(c, c.thr_tiles))) return rc;
    if (c.mg_max_lb > 0 && (rc = mg_lists_for(c, active))) return rc;
    return RECON_OK;
}

int solver_init_slots(Ctx& c, const std::vector<int>& slots, const float* lo, const float* hi) {
    if (slots.empty()) return RECON_OK;
    lists_for(c, slots, &c.tmp_tiles, nullptr, nullptr);
    int rc;
    if ((rc = fill_list(c, c.tmp_tiles))) return rc;
    // the slot list itself rides in the tmp list's counter buffer (one int per slot)
    RECON_CUDA(cudaMemcpyAsync(c.tmp_tiles.counters, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice,
                               c.stream));
    k_reset_slots<<<((int)slots.size() + 127) / 128, 128, 0, c.stream>>>(
        reinterpret_cast<const int*>(c.tmp_tiles.counters), (int)slots.size(), c.d_const, c.d_state);
    RECON_CUDA(cudaMemsetAsync(c.tmp_tiles.counters, 0, sizeof(unsigned) * c.n, c.stream));
    const ItemList L = c.tmp_tiles.view();
    const int grid = grid_for(c, L.n_items);
    if (c.precision == 1) {
        k_load<float><<<grid, kStencilThreads, 0, c.stream>>>(L, c.d_geom, c.d_const, lo, hi,
                                                             static_cast<float*>(c.field[RECON_F_MUL]),
                                                             static_cast<float*>(c.field[RECON_F_MUH]));
        k_init<float><<<grid, kStencilThreads, 0, c.stream>>>(L, c.d_geom, c.d_const, ptrs<float>(c));
    } else {
        k_load<double><<<grid, kStencilThreads, 0, c.stream>>>(L, c.d_geom, c.d_const, lo, hi,
                                                              static_cast<double*>(c.field[RECON_F_MUL]),
                                                              static_cast<double*>(c.field[RECON_F_MUH]));
        k_init<double><<<grid, kStencilThreads, 0, c.stream>>>(L, c.d_geom, c.d_const, ptrs<double>(c));
    }
    c.launches += 3;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

int solver_extract_slots(Ctx& c, const std::vector<int>& slots, float* Z, float* rhoe) {
    if (slots.empty()) return RECON_OK;
    lists_for(c, slots, &c.tmp_tiles, nullptr, nullptr);
    int rc;
    if ((rc = fill_list(c, c.tmp_tiles))) return rc;
    const ItemList L = c.tmp_tiles.view();
    const int grid = grid_for(c, L.n_items);
    if (c.precision == 1)
        k_extract<float><<<grid, kStencilThreads, 0, c.stream>>>(L, c.d_geom, ptrs<float>(c), Z, rhoe, nullptr,
                                                                 nullptr, water_z(), z_exponent());
    else
        k_extract<double><<<grid, kStencilThreads, 0, c.stream>>>(L, c.d_geom, ptrs<double>(c), Z, rhoe, nullptr,
                                                                  nullptr, water_z(), z_exponent());
    c.launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
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
        for (int f = 0; f < KF_COUNT; ++f) bytes[f] = h[f] + c.host_acct[f];
    for (int f = 0; f < KF_COUNT; ++f) c.host_acct[f] = 0;
    return RECON_OK;
}

int solver_read_state(Ctx& c, std::vector<SliceState>& out) {
    out.resize(c.n);
    RECON_CUDA(cudaMemcpyAsync(out.data(), c.d_state, sizeof(SliceState) * c.n, cudaMemcpyDeviceToHost, c.stream));
    RECON_CUDA(cudaStreamSynchronize(c.stream));
    return RECON_OK;
}

}  // namespace recon
