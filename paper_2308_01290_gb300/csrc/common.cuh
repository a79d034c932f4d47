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
    int cluster;               // 1: the Z^m solve of this slice runs in the cluster kernel
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
};

// Mutable per-slice state (device).
struct SliceState {
    double beta, beta_t, thr_d;   // beta, beta~, lambda/beta
    float thr_f;                  // lambda/beta rounded to float (decisions)
    int k;                        // iterations done
    int active;                   // k < iters
    // PCG of the Z^m step
    int cg_it, cg_done;
    double abar2, bb, rr, rr0, ry, pq, alpha, betacg;
    // statistics of the last iteration (eq. obj_unconstraint terms)
    double stat[6];               // fid_L, fid_H, mod_1, mod_2, relax_sum (unscaled), unused
    long long nnz[4];
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
    KF_PCG_CLUSTER,
    KF_FCG,
    KF_PROJ,
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
