// Device-side types shared by the solver kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace recon {

template <typename T>
struct cplx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) {
    return {a.x - b.x, a.y - b.y};
}

// Geometry and memory placement of one slice inside the batch pools.
struct SliceGeom {
    int nx, ny, pitch;   // real fields: ny rows of pitch elements
    int nh, cpitch;      // spectra: ny rows of cpitch complex, nh = nx/2 + 1 used
    long long off;       // element offset of the slice in every real field pool
    long long coff;      // element offset of the slice in every spectrum pool
    long long ext_off;   // element offset of the slice in unpadded caller buffers
    unsigned plan_x, plan_y;   // FFT plans (radix sequences) along x and y
    long long twx, twy;        // offsets of the twiddle tables exp(-2 pi i t/N) in the twiddle pool
    long long symx, symy;      // offsets of the tables 4 sin^2(pi t/N) in the symbol pool
    int rows_per_item, cols_per_item;
    float inv_n;               // 1 / (nx ny) rounded to float (spectral scale of the FP32 transforms)
    int lvl;                   // multigrid level of this grid (0: the slice's own grid)
};

// Model constants that the FP32 kernels read, by index: each is one FP64
// expression of the SliceConst fields (kc_value), rounded to float once on
// the host into SliceConst::fk.  GB300 issues FP64 at a small fraction of its
// FP32 rate, so the FP32 kernels never convert or divide doubles per thread;
// the rounded values are the same floats a per-thread conversion would give.
enum KConst {
    KC_A00, KC_A01, KC_A10, KC_A11,   // a[k][i]
    KC_B00, KC_B01, KC_B10, KC_B11,   // b[k][j]
    KC_P1, KC_P2, KC_PSI1, KC_PSI2,
    KC_R, KC_C12, KC_INV_CRHO, KC_INV_AW,
    KC_CF1, KC_CF2,                   // c_f1, c_f2 (f-update diagonals)
    KC_SINO_AG, KC_SINO_BC,           // domain 1: cross / gamma, c12 - cross
    KC_SINO_D0, KC_SINO_D1,           // domain 1: alpha_k + c'_k
    KC_SINO_AL0, KC_SINO_AL1,         // domain 1: alpha_k / gamma
    KC_SINO_CP0, KC_SINO_CP1,         // domain 1: c'_k
    KC_N
};

// Model constants and parameters of one slice (FP64, read-only on device).
struct SliceConst {
    double a00, a01, a10, a11;   // a[k][i]: basis k at arm i (L, H)
    double b00, b01, b10, b11;   // b[k][j]: basis k at E_j
    double P1, P2, psi1, psi2;
    double r, c_f1, c_f2, c12, c_rho, a_w, det;
    double inv_S, zclip_hi, rho_air;
    double lambda, beta0, kappa, tau;
    double cg_tol;
    // sinogram-domain data terms (domain 1): alpha_k = sum_i a[k][i]^2,
    // c'_k = sum_j b[k][j]^2, cross = sum_i a[0][i] a[1][i], 1/gamma
    double fa0, fa1, fcp0, fcp1, fcross, inv_gamma;
    int iters, order, cg_max, domain;
    int gn;                       // domain 2: per-ray Gauss-Newton weights replace alpha_k and the cross term
    float fk[KC_N];               // kc_value(*this, i) rounded to float (set by finish_const)
};

// The FP64 value of model constant `id` of slice constants c.
__host__ __device__ inline double kc_value(const SliceConst& c, int id) {
    switch (id) {
        case KC_A00: return c.a00;
        case KC_A01: return c.a01;
        case KC_A10: return c.a10;
        case KC_A11: return c.a11;
        case KC_B00: return c.b00;
        case KC_B01: return c.b01;
        case KC_B10: return c.b10;
        case KC_B11: return c.b11;
        case KC_P1: return c.P1;
        case KC_P2: return c.P2;
        case KC_PSI1: return c.psi1;
        case KC_PSI2: return c.psi2;
        case KC_R: return c.r;
        case KC_C12: return c.c12;
        case KC_INV_CRHO: return 1.0 / c.c_rho;
        case KC_INV_AW: return 1.0 / c.a_w;
        case KC_CF1: return c.c_f1;
        case KC_CF2: return c.c_f2;
        case KC_SINO_AG: return c.gn ? 0.0 : c.fcross * c.inv_gamma;
        case KC_SINO_BC: return c.c12 - c.fcross;
        case KC_SINO_D0: return c.fa0 + c.fcp0;
        case KC_SINO_D1: return c.fa1 + c.fcp1;
        case KC_SINO_AL0: return c.gn ? c.inv_gamma : c.fa0 * c.inv_gamma;
        case KC_SINO_AL1: return c.gn ? c.inv_gamma : c.fa1 * c.inv_gamma;
        case KC_SINO_CP0: return c.fcp0;
        case KC_SINO_CP1: return c.fcp1;
        default: return 0.0;
    }
}

// Fill the float copies of the model constants (host, after any change of
// the FP64 fields).
inline void finish_const(SliceConst& c) {
    for (int i = 0; i < KC_N; ++i) c.fk[i] = (float)kc_value(c, i);
}

// Model constant `id` in the kernel's precision: the host-rounded float for
// FP32 kernels, the FP64 expression itself for FP64 kernels.
template <typename T>
__device__ __forceinline__ T kc(const SliceConst& c, int id);
template <>
__device__ __forceinline__ float kc<float>(const SliceConst& c, int id) {
    return c.fk[id];
}
template <>
__device__ __forceinline__ double kc<double>(const SliceConst& c, int id) {
    return kc_value(c, id);
}

// Mutable per-slice state (device).
struct SliceState {
    double beta, beta_t, thr_d;   // beta, beta~, lambda/beta
    float thr_f;                  // lambda/beta rounded to float (decisions)
    int k;                        // iterations done
    int active;                   // k < iters
    // PCG of the Z^m step
    int cg_it, cg_done;
    double abar2, bb, rr, rr0, ry, pq, alpha, betacg;
    // float roundings of the scalars the FP32 kernels read per item, written
    // by the one thread that writes the FP64 value (set_* below):
    // beta, beta~, 4 beta~, abar^2, sqrt(abar^2 + 4 beta~), alpha, beta_cg
    float beta_f, beta_t_f, b4_f, abar2_f, rnum_f, alpha_f, betacg_f;
    // statistics of the last iteration (eq. obj_unconstraint terms)
    double stat[6];               // fid_L, fid_H, mod_1, mod_2, relax_sum (unscaled), unused
    long long nnz[4];
};

// Writers of the scalars that have float copies (one thread each).
__device__ __forceinline__ void set_beta(SliceState& st, double beta, const SliceConst& c) {
    st.beta = beta;
    st.beta_t = c.tau * beta;
    st.thr_d = c.lambda / beta;
    st.thr_f = (float)st.thr_d;
    st.beta_f = (float)beta;
    st.beta_t_f = (float)st.beta_t;
    st.b4_f = (float)(4.0 * st.beta_t);
}
__device__ __forceinline__ void set_abar2(SliceState& st, double abar2) {
    st.abar2 = abar2;
    st.abar2_f = (float)abar2;
    st.rnum_f = (float)sqrt(abar2 + 4.0 * st.beta_t);
}
__device__ __forceinline__ void set_alpha(SliceState& st, double alpha) {
    st.alpha = alpha;
    st.alpha_f = (float)alpha;
}
__device__ __forceinline__ void set_betacg(SliceState& st, double betacg) {
    st.betacg = betacg;
    st.betacg_f = (float)betacg;
}

// Per-slice scalars in the kernel's precision: the float copies for FP32
// kernels, the FP64 values (and expressions of them) for FP64 kernels.
template <typename T>
struct Sc;
template <>
struct Sc<float> {
    static __device__ __forceinline__ float beta(const SliceState& s) { return s.beta_f; }
    static __device__ __forceinline__ float beta_t(const SliceState& s) { return s.beta_t_f; }
    static __device__ __forceinline__ float b4(const SliceState& s) { return s.b4_f; }
    static __device__ __forceinline__ float abar2(const SliceState& s) { return s.abar2_f; }
    static __device__ __forceinline__ float rnum(const SliceState& s) { return s.rnum_f; }
    static __device__ __forceinline__ float alpha(const SliceState& s) { return s.alpha_f; }
    static __device__ __forceinline__ float betacg(const SliceState& s) { return s.betacg_f; }
};
template <>
struct Sc<double> {
    static __device__ __forceinline__ double beta(const SliceState& s) { return s.beta; }
    static __device__ __forceinline__ double beta_t(const SliceState& s) { return s.beta_t; }
    static __device__ __forceinline__ double b4(const SliceState& s) { return 4.0 * s.beta_t; }
    static __device__ __forceinline__ double abar2(const SliceState& s) { return s.abar2; }
    static __device__ __forceinline__ double rnum(const SliceState& s) { return sqrt(s.abar2 + 4.0 * s.beta_t); }
    static __device__ __forceinline__ double alpha(const SliceState& s) { return s.alpha; }
    static __device__ __forceinline__ double betacg(const SliceState& s) { return s.betacg; }
};

// A unit of work: one tile / row group / column group of one slice.
struct Item {
    int slice, a, b, c;
};

// Item list of one kernel family with per-slice item ranges and the scratch
// used by the "last item of the slice reduces" pattern.
struct ItemList {
    const Item* items;
    int n_items;
    const int* lo;            // first item of slice s
    const int* cnt;           // number of items of slice s
    double* partials;         // n_items * kMaxPartials
    unsigned int* counters;   // one per slice (returned to zero after use)
};

// Kernel families for timing and algorithmic-byte accounting.
enum KFam {
    KF_THR_RHS = 0,
    KF_ROWS_FWD,
    KF_COLS,
    KF_ROWS_INV,
    KF_SYNTH,
    KF_CG_INIT,
    KF_PCG_FWD,
    KF_COLS_PRE,
    KF_PCG_INV,
    KF_FCG,
    KF_PROJ,
    KF_MG_FWD,      // multigrid PCG: update, convergence test, first restriction
    KF_MG_Y,        // multigrid PCG: fine-level correction and smoothing, r.y
    KF_MG_PQ,       // multigrid PCG: new direction p, q = M p, p.q
    KF_MG_LEVELS,   // multigrid PCG: the coarse tile levels (restriction and correction passes)
    KF_MG_BLOCK,    // multigrid PCG: the in-block levels of every slice and the coarsest solve
    KF_MG_SETUP,    // multigrid PCG: a^2 of the levels and the coarsest inverse (once per Z^m solve)
    KF_OTHER,
    KF_COUNT
};

constexpr int kMaxPartials = 12;
constexpr int kTileW = 64;       // tiles are kTileW pixels wide; their height is TileDim<T>::TH
constexpr int kTileHFloat = 32;
constexpr int kTileHDouble = 16;
constexpr int kStencilThreads = 256;
constexpr int kFftThreads = 256;
constexpr int kFftMinBlocks = 3;   // resident blocks per SM the FFT kernels are compiled for
// complex elements one FFT block transforms at a time (rows or columns)
template <typename T>
struct FftBudget;
template <>
struct FftBudget<float> {
    static constexpr int E = 4096;
};
template <>
struct FftBudget<double> {
    static constexpr int E = 2048;
};

// Copy a small struct into shared memory (whole block), no sync.
template <typename S>
__device__ __forceinline__ void stage_struct(S* dst, const S* src) {
    static_assert(sizeof(S) % 4 == 0, "");
    for (int i = threadIdx.x; i < (int)(sizeof(S) / 4); i += blockDim.x)
        reinterpret_cast<int*>(dst)[i] = __ldg(reinterpret_cast<const int*>(src) + i);
}

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Block-wide sum of NV doubles; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* NV * 32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q * 32 + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[q * 32 + w];
            v[q] = s;
        }
    }
    __syncthreads();
}

// Compensated (float-float) addition: (h, l) += (h2, l2), additions only.
__device__ __forceinline__ void ff_add(float& h, float& l, float h2, float l2) {
    const float s = h + h2;
    const float bb = s - h;
    float e = (h - (s - bb)) + (h2 - bb);   // exact error of s (two-sum)
    e += l + l2;
    h = s + e;
    l = e - (h - s);
}

// Block-wide sum of the NV per-thread partials x of a kernel computing in
// T; result in thread 0.  FP32 kernels sum in compensated float-float
// arithmetic (across each warp, then across the warps), which runs on the
// FP32 pipes (GB300 issues FP64 at a small fraction of the FP32 rate), and
// convert once to FP64; FP64 kernels sum in FP64.
template <typename T, int NV>
__device__ __forceinline__ void block_sum_t(const T (&x)[NV], double (&v)[NV], double* sh /* NV * 32 */) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = (double)x[q];
        block_sum<NV>(v, sh);
    } else {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
        float* shf = reinterpret_cast<float*>(sh);   // (h, l) per warp: NV * 64 floats
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float h = (float)x[q], l = 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_down_sync(0xffffffffu, h, o);
                const float l2 = __shfl_down_sync(0xffffffffu, l, o);
                ff_add(h, l, h2, l2);
            }
            if (lane == 0) {
                shf[q * 64 + 2 * warp] = h;
                shf[q * 64 + 2 * warp + 1] = l;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // the warp sums in float-float too; one conversion to FP64 per value
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                float h = 0.f, l = 0.f;
                for (int w = 0; w < nw; ++w) ff_add(h, l, shf[q * 64 + 2 * w], shf[q * 64 + 2 * w + 1]);
                v[q] = (double)h + (double)l;
            }
        }
        __syncthreads();
    }
}

// Store the partials of one item; returns true (in thread 0 only) when this
// item is the last of its slice to finish, in which case `tot` holds the sum
// of all partials of the slice in a fixed order (deterministic).  The final
// sum is taken by the whole block: each thread adds a strided subset of the
// partials (read through L2), then a block reduction in fixed order.
template <int NV>
__device__ __forceinline__ bool item_reduce(const ItemList& L, int item, int slice, const double (&v)[NV],
                                            double (&tot)[NV], double* sh /* NV * 32 */) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) L.partials[(size_t)item * kMaxPartials + q] = v[q];
        __threadfence();
        const unsigned prev = atomicAdd(&L.counters[slice], 1u);
        s_last = (prev == (unsigned)L.cnt[slice] - 1u) ? 1 : 0;
    }
    __syncthreads();
    const int last = s_last;
    if (!last) return false;
    __threadfence();
    const int lo = L.lo[slice], n = L.cnt[slice];
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(L.partials + (size_t)(lo + i) * kMaxPartials + q);
    }
    block_sum<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) tot[q] = acc[q];
        L.counters[slice] = 0u;
    }
    return threadIdx.x == 0;
}

}  // namespace recon
