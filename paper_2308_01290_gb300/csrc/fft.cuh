// Shared-memory mixed-radix (2, 3, 4, 5, 7, 8) Stockham FFT for a batch of
// sequences of the same length N held in shared memory.
//
// Stage with radix R and current sub-transform size Ns (product of the
// radices already applied, starting at 1): for butterfly j in [0, N/R),
// k = j mod Ns, read x[j + r N/R] (r < R), multiply by w^(r k N/(Ns R)) with
// w = exp(-+2 pi i / N), take an R-point DFT, and write
// x'[(j / Ns) Ns R + k + r Ns].  After the last stage the result is in
// natural order (Stockham autosort).  Stages ping-pong between two shared
// buffers, one butterfly per thread at a time.  Element i of a sequence lives
// at slot i + i/8 (one pad slot every 8) so that the stride-R accesses of
// the early stages do not pile up in one shared-memory bank.
#pragma once
#include "common.cuh"

namespace recon {

// Radices of the stages, 4 bits each from the low end; the stage count in
// bits 28..31.  Powers of two first (8, then 4, then 2), then 3, 5, 7.
__host__ __device__ inline unsigned fft_plan_code(int n) {
    unsigned code = 0;
    int ns = 0;
    int m = n;
    auto push = [&](int r) {
        code |= (unsigned)r << (4 * ns);
        ++ns;
    };
    while (m % 8 == 0) { push(8); m /= 8; }
    while (m % 4 == 0) { push(4); m /= 4; }
    while (m % 2 == 0) { push(2); m /= 2; }
    while (m % 3 == 0) { push(3); m /= 3; }
    while (m % 5 == 0) { push(5); m /= 5; }
    while (m % 7 == 0) { push(7); m /= 7; }
    return code | ((unsigned)ns << 28);
}

__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
// slots a padded sequence of n elements occupies
__host__ __device__ inline int padded_len(int n) { return n + (n >> 3) + 1; }

// n / d for 0 <= n < 2^24 using a float reciprocal and one correction.
__device__ __forceinline__ int fdiv(int n, int d, float inv_d) {
    int q = (int)((float)n * inv_d);
    q -= (q * d > n) ? 1 : 0;
    q += ((q + 1) * d <= n) ? 1 : 0;
    return q;
}

// multiply by -i (forward) or +i (inverse)
template <typename T>
__device__ __forceinline__ cplx<T> rot90(cplx<T> a, int dir) {
    return dir < 0 ? cplx<T>{a.y, -a.x} : cplx<T>{-a.y, a.x};
}

template <typename T>
__device__ __forceinline__ void dft2(cplx<T>* v) {
    const cplx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <typename T>
__device__ __forceinline__ void dft4(cplx<T>* v, int dir) {
    const cplx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const cplx<T> t2 = cadd(v[1], v[3]), t3 = rot90(csub(v[1], v[3]), dir);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}

template <typename T>
__device__ __forceinline__ void dft8(cplx<T>* v, int dir) {
    const T h = T(0.70710678118654752440);
    cplx<T> a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = cadd(v[k], v[k + 4]);
        b[k] = csub(v[k], v[k + 4]);
    }
    // b1 *= w8^1, b2 *= w8^2, b3 *= w8^3 with w8 = exp(dir i pi / 4)
    {
        const cplx<T> x = b[1];
        b[1] = dir < 0 ? cplx<T>{h * (x.x + x.y), h * (x.y - x.x)} : cplx<T>{h * (x.x - x.y), h * (x.y + x.x)};
        b[2] = rot90(b[2], dir);
        const cplx<T> y = b[3];
        b[3] = dir < 0 ? cplx<T>{h * (y.y - y.x), -h * (y.x + y.y)} : cplx<T>{-h * (y.x + y.y), h * (y.x - y.y)};
    }
    dft4(a, dir);
    dft4(b, dir);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        v[2 * m] = a[m];
        v[2 * m + 1] = b[m];
    }
}

// Direct R-point DFT for the odd radices 3, 5, 7 (constants cos, sin of
// 2 pi m / R from a small table).
template <typename T, int R>
__device__ __forceinline__ void dft_odd(cplx<T>* v, int dir) {
    // cos(2 pi m / R), sin(2 pi m / R) for m < R
    constexpr double c3[3] = {1.0, -0.5, -0.5};
    constexpr double s3[3] = {0.0, 0.86602540378443864676, -0.86602540378443864676};
    constexpr double c5[5] = {1.0, 0.30901699437494742410, -0.80901699437494742410, -0.80901699437494742410,
                              0.30901699437494742410};
    constexpr double s5[5] = {0.0, 0.95105651629515357212, 0.58778525229247312917, -0.58778525229247312917,
                              -0.95105651629515357212};
    constexpr double c7[7] = {1.0,
                              0.62348980185873353053,
                              -0.22252093395631440429,
                              -0.90096886790241912624,
                              -0.90096886790241912624,
                              -0.22252093395631440429,
                              0.62348980185873353053};
    constexpr double s7[7] = {0.0,
                              0.78183148246802980871,
                              0.97492791218182360702,
                              0.43388373911755812048,
                              -0.43388373911755812048,
                              -0.97492791218182360702,
                              -0.78183148246802980871};
    cplx<T> out[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        cplx<T> acc = v[0];
#pragma unroll
        for (int n = 1; n < R; ++n) {
            const int m = (n * k) % R;
            const T c = T(R == 3 ? c3[m] : (R == 5 ? c5[m] : c7[m]));
            const T sv = T(R == 3 ? s3[m] : (R == 5 ? s5[m] : s7[m]));
            const T s = dir < 0 ? -sv : sv;
            acc.x += v[n].x * c - v[n].y * s;
            acc.y += v[n].x * s + v[n].y * c;
        }
        out[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <typename T, int R>
__device__ __forceinline__ void dft(cplx<T>* v, int dir) {
    if (R == 2) dft2(v);
    else if (R == 4) dft4(v, dir);
    else if (R == 8) dft8(v, dir);
    else dft_odd<T, R>(v, dir);
}

// Integer n / d and n % d for the index maps of a stage: shifts when d is a
// power of two, else a float reciprocal with one correction (n < 2^24).
struct DivMod {
    int d, shift;
    float inv;
    __device__ __forceinline__ explicit DivMod(int dd) : d(dd), shift(-1), inv(1.0f / (float)dd) {
        if ((dd & (dd - 1)) == 0) shift = __ffs(dd) - 1;
    }
    __device__ __forceinline__ int div(int n) const { return shift >= 0 ? (n >> shift) : fdiv(n, d, inv); }
};

// One stage from buffer `in` to buffer `out` (sequence b at +b*ld, padded
// indexing), one butterfly per thread at a time.
template <typename T, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int N, int Ns,
                                          int batch, int ld, const cplx<T>* __restrict__ tw, int dir) {
    const int nbf = N / R;
    const int total = batch * nbf;
    const int step = N / (Ns * R);
    const DivMod dn(nbf), ds(Ns);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int b = dn.div(t), j = t - b * nbf;
        const int jn = ds.div(j), k = j - jn * Ns;
        const cplx<T>* src = in + b * ld;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[pad8(j + r * nbf)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                cplx<T> w = tw[r * k * step];
                if (dir > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft<T, R>(v, dir);
        cplx<T>* dst = out + b * ld;
        const int idxD = jn * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[pad8(idxD + r * Ns)] = v[r];
    }
}

// Transform `batch` sequences of length N (dir -1 forward, +1 inverse,
// unnormalised), ping-ponging between buffers a and b; returns the buffer
// holding the result.  `plan` from fft_plan_code(N); tw[t] = exp(-2 pi i t/N)
// in global memory.  The caller synchronises before (data ready); the
// function synchronises after every stage.
template <typename T>
__device__ __forceinline__ cplx<T>* fft_batch(cplx<T>* a, cplx<T>* b, int N, unsigned plan, int batch, int ld,
                                              const cplx<T>* tw, int dir) {
    const int ns = (int)(plan >> 28);
    int Ns = 1;
    cplx<T>* in = a;
    cplx<T>* out = b;
    for (int s = 0; s < ns; ++s) {
        const int R = (int)((plan >> (4 * s)) & 15u);
        switch (R) {
            case 8: fft_stage<T, 8>(in, out, N, Ns, batch, ld, tw, dir); break;
            case 4: fft_stage<T, 4>(in, out, N, Ns, batch, ld, tw, dir); break;
            case 2: fft_stage<T, 2>(in, out, N, Ns, batch, ld, tw, dir); break;
            case 3: fft_stage<T, 3>(in, out, N, Ns, batch, ld, tw, dir); break;
            case 5: fft_stage<T, 5>(in, out, N, Ns, batch, ld, tw, dir); break;
            default: fft_stage<T, 7>(in, out, N, Ns, batch, ld, tw, dir); break;
        }
        __syncthreads();
        cplx<T>* t = in;
        in = out;
        out = t;
        Ns *= R;
    }
    return in;
}

// ---------------------------------------------------------------------------
// Compile-time power-of-two transforms.  Same Stockham stages as above (8s
// first, then one 4 or 2), but every index map is a shift or a mask, the
// padded shared-memory offsets of a butterfly's R legs are immediates, and
// a stage's source or destination may be a functor that reads or writes HBM
// directly, so the first and last stages of an item need no separate copy
// through shared memory.
// ---------------------------------------------------------------------------

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ constexpr bool is_pow2c(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Leading dimension (complex slots) of one column sequence of length N in
// the column pass.  Power-of-two N >= 64 takes padded_len(N) + 1, which is
// 2 mod 16 slots: the eight columns of a column-fastest access then fall in
// distinct banks.  Other N take the odd length padded_len(N) | 1.
__host__ __device__ inline int col_ld(int n) {
    return (is_pow2c(n) && n >= 64) ? padded_len(n) + 1 : (padded_len(n) | 1);
}

__host__ __device__ constexpr int count_factor(int n, int f) { return (n > 0 && n % f == 0) ? 1 + count_factor(n / f, f) : 0; }

// Stage plan of a compile-time length N = 2^a 3^b 5^c 7^d: radix-8 stages,
// then one 4 or 2, then 3s, 5s, 7s (the order of fft_plan_code).  Stage
// s > 0 multiplies leg r of butterfly k (k < ns) by w^r,
// w = exp(-+2 pi i k / (ns R)).  Its twiddles sit in a stage-major table that
// follows the N-entry table exp(-2 pi i t/N) in the twiddle pool: for each
// stage s > 0, blocks of ns entries contiguous in k holding w, w^2 and w^4
// as far as they are below R (R = 2, 4, 8; the butterfly forms w^3, w^5, w^6,
// w^7 as products of two of them), or w .. w^(R-1) (R = 3, 5, 7).
template <int N>
struct P2Plan {
    static constexpr int L = count_factor(N, 2);
    static constexpr int N8 = L / 3;                      // radix-8 stages
    static constexpr int REM = L - 3 * N8;                // 0, 1 (radix 2) or 2 (radix 4)
    static constexpr int P2S = N8 + (REM ? 1 : 0);        // power-of-two stages
    static constexpr int C3 = count_factor(N, 3), C5 = count_factor(N, 5), C7 = count_factor(N, 7);
    static constexpr int S = P2S + C3 + C5 + C7;          // stage count
    __host__ __device__ static constexpr int radix(int s) {
        return s < N8 ? 8 : (s < P2S ? (REM == 2 ? 4 : 2) : (s < P2S + C3 ? 3 : (s < P2S + C3 + C5 ? 5 : 7)));
    }
    __host__ __device__ static constexpr int ns(int s) { return s == 0 ? 1 : ns(s - 1) * radix(s - 1); }
    // stored powers per butterfly
    __host__ __device__ static constexpr int powers(int s) {
        return radix(s) == 8 ? 3 : (radix(s) == 4 ? 2 : (radix(s) == 2 ? 1 : radix(s) - 1));
    }
    __host__ __device__ static constexpr int tw_off(int s) {
        return s <= 1 ? 0 : tw_off(s - 1) + powers(s - 1) * ns(s - 1);
    }
};

// Sources and destinations of a stage provide load_legs<R, NBF>(b, j, v)
// (v[r] = element j + r NBF of sequence b) and store_legs<R, NS>(b, idx0, v)
// (element idx0 + r NS of sequence b = v[r]).

// Shared-memory sequence set: sequence b at p + b * ld, padded indexing.
// With the radix-8-first plans NBF and NS are 1 or multiples of 8 (and with
// NS = 1, idx0 is a multiple of R, R | 8), so the padded offsets of the legs
// are immediates.
template <typename T>
struct SmemSeq {
    cplx<T>* p;
    int ld;
    template <int R, int NBF>
    __device__ __forceinline__ void load_legs(int b, int j, cplx<T>* v) const {
        const cplx<T>* s = p + b * ld;
        if constexpr (NBF % 8 == 0) {
            const int o = pad8(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[o + r * (NBF + NBF / 8)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[pad8(j + r * NBF)];
        }
    }
    template <int R, int NS>
    __device__ __forceinline__ void store_legs(int b, int idx0, const cplx<T>* v) const {
        cplx<T>* s = p + b * ld;
        if constexpr (NS == 1 && 8 % R == 0) {
            const int o = pad8(idx0);
#pragma unroll
            for (int r = 0; r < R; ++r) s[o + r] = v[r];
        } else if constexpr (NS % 8 == 0) {
            const int o = pad8(idx0);
#pragma unroll
            for (int r = 0; r < R; ++r) s[o + r * (NS + NS / 8)] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) s[pad8(idx0 + r * NS)] = v[r];
        }
    }
};

// Element-wise functor source f(b, idx) -> cplx and destination f(b, idx, v).
template <typename T, class F>
struct FnLoad {
    F f;
    template <int R, int NBF>
    __device__ __forceinline__ void load_legs(int b, int j, cplx<T>* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = f(b, j + r * NBF);
    }
};
template <typename T, class F>
struct FnStore {
    F f;
    template <int R, int NS>
    __device__ __forceinline__ void store_legs(int b, int idx0, const cplx<T>* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) f(b, idx0 + r * NS, v[r]);
    }
};
template <typename T, class F>
__device__ __forceinline__ FnLoad<T, F> fn_load(F f) {
    return FnLoad<T, F>{f};
}
template <typename T, class F>
__device__ __forceinline__ FnStore<T, F> fn_store(F f) {
    return FnStore<T, F>{f};
}

// v * w (DIR < 0) or v * conj(w) (DIR > 0)
template <typename T, int DIR>
__device__ __forceinline__ cplx<T> cmul_dir(cplx<T> v, cplx<T> w) {
    if constexpr (DIR < 0) return {v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x};
    else return {v.x * w.x + v.y * w.y, v.y * w.x - v.x * w.y};
}

// Stage s of the length-N plan over `batch` sequences.  Tasks map to
// (sequence b, butterfly j) with j fastest, or with b fastest over CB slots
// (BFAST: tasks with b >= batch idle), which keeps a column-fastest HBM
// access coalesced.
template <typename T, int N, int STAGE, int DIR, bool BFAST, int CB, class SRC, class DST>
__device__ __forceinline__ void p2_stage(int batch, const cplx<T>* __restrict__ tw, const SRC& src, const DST& dst) {
    constexpr int R = P2Plan<N>::radix(STAGE);
    constexpr int NS = P2Plan<N>::ns(STAGE);
    constexpr int NBF = N / R;
    const int total = BFAST ? CB * NBF : batch * NBF;
#pragma unroll 1
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int b, j;
        if constexpr (BFAST) {
            b = t % CB;
            j = t / CB;
            if (b >= batch) continue;
        } else {
            j = t % NBF;
            b = t / NBF;
        }
        cplx<T> v[R];
        src.template load_legs<R, NBF>(b, j, v);
        const int k = j % NS;
        if constexpr (NS > 1) {
            const cplx<T>* t = tw + P2Plan<N>::tw_off(STAGE) + k;
            const cplx<T> w1 = t[0];
            if constexpr (R == 2) {
                v[1] = cmul_dir<T, DIR>(v[1], w1);
            } else if constexpr (R % 2 == 1) {
                v[1] = cmul_dir<T, DIR>(v[1], w1);
#pragma unroll
                for (int r = 2; r < R; ++r) v[r] = cmul_dir<T, DIR>(v[r], t[(r - 1) * NS]);
            } else {
                const cplx<T> w2 = t[NS];
                if constexpr (R == 4) {
                    v[1] = cmul_dir<T, DIR>(v[1], w1);
                    v[2] = cmul_dir<T, DIR>(v[2], w2);
                    v[3] = cmul_dir<T, DIR>(v[3], cmul(w1, w2));
                } else {
                    const cplx<T> w4 = t[2 * NS];
                    const cplx<T> w3 = cmul(w1, w2);
                    v[1] = cmul_dir<T, DIR>(v[1], w1);
                    v[2] = cmul_dir<T, DIR>(v[2], w2);
                    v[3] = cmul_dir<T, DIR>(v[3], w3);
                    v[4] = cmul_dir<T, DIR>(v[4], w4);
                    v[5] = cmul_dir<T, DIR>(v[5], cmul(w1, w4));
                    v[6] = cmul_dir<T, DIR>(v[6], cmul(w2, w4));
                    v[7] = cmul_dir<T, DIR>(v[7], cmul(w3, w4));
                }
            }
        }
        dft<T, R>(v, DIR);
        dst.template store_legs<R, NS>(b, (j / NS) * NS * R + k, v);
    }
}

// Stages FIRST..LAST between the shared buffers a and b (ping-pong, stage
// FIRST reads a), j-fastest; a synchronisation after each stage.  Returns
// the buffer holding the result.
template <typename T, int N, int DIR, int FIRST, int LAST>
__device__ __forceinline__ cplx<T>* p2_smem_stages(cplx<T>* a, cplx<T>* b, int ld, int batch, const cplx<T>* tw) {
    if constexpr (FIRST > LAST) {
        return a;
    } else {
        p2_stage<T, N, FIRST, DIR, false, 1>(batch, tw, SmemSeq<T>{a, ld}, SmemSeq<T>{b, ld});
        __syncthreads();
        return p2_smem_stages<T, N, DIR, FIRST + 1, LAST>(b, a, ld, batch, tw);
    }
}

}  // namespace recon
