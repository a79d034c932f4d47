// Shared-memory mixed-radix (2, 3, 4, 5, 7, 8) Stockham FFT for a batch of
// sequences of the same length N held in shared memory.
//
// Stage s with radix R and current sub-transform size Ns (product of the
// radices already applied, starting at 1): for butterfly j in [0, N/R),
// k = j mod Ns, read in[j + r N/R] (r < R), multiply by w^(r k N/(Ns R)) with
// w = exp(-+2 pi i / N), take an R-point DFT, and write
// out[(j / Ns) Ns R + k + r Ns].  The result is in natural order after the
// last stage (Stockham autosort; no bit reversal).
#pragma once
#include "common.cuh"

namespace recon {

struct FftPlan {
    int n, ns;
    int radix[24];
};

__device__ __forceinline__ FftPlan make_plan(int n) {
    FftPlan p;
    p.n = n;
    p.ns = 0;
    int m = n;
    while (m % 8 == 0) { p.radix[p.ns++] = 8; m /= 8; }
    while (m % 4 == 0) { p.radix[p.ns++] = 4; m /= 4; }
    while (m % 2 == 0) { p.radix[p.ns++] = 2; m /= 2; }
    while (m % 3 == 0) { p.radix[p.ns++] = 3; m /= 3; }
    while (m % 5 == 0) { p.radix[p.ns++] = 5; m /= 5; }
    while (m % 7 == 0) { p.radix[p.ns++] = 7; m /= 7; }
    return p;
}

template <typename T>
__device__ __forceinline__ void sincospi_t(T x, T* s, T* c);
template <>
__device__ __forceinline__ void sincospi_t<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void sincospi_t<double>(double x, double* s, double* c) { sincospi(x, s, c); }

// tw[t] = exp(-2 pi i t / n), t < n (forward roots).
template <typename T>
__device__ __forceinline__ void fill_twiddles(cplx<T>* tw, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        T s, c;
        // angle 2 t / n in units of pi; reduce to keep the argument small
        sincospi_t<T>(T(2) * T(t) / T(n), &s, &c);
        tw[t] = {c, -s};
    }
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

// Direct R-point DFT for odd radices 3, 5, 7.
template <typename T, int R>
__device__ __forceinline__ void dft_odd(cplx<T>* v, int dir) {
    cplx<T> out[R];
    T cs[R], sn[R];
#pragma unroll
    for (int m = 0; m < R; ++m) sincospi_t<T>(T(2 * m) / T(R), &sn[m], &cs[m]);
#pragma unroll
    for (int k = 0; k < R; ++k) {
        cplx<T> acc = v[0];
#pragma unroll
        for (int n = 1; n < R; ++n) {
            const int m = (n * k) % R;
            const T c = cs[m], s = dir < 0 ? -sn[m] : sn[m];
            acc.x += v[n].x * c - v[n].y * s;
            acc.y += v[n].x * s + v[n].y * c;
        }
        out[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <typename T, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int N, int Ns,
                                          int batch, int ld, const cplx<T>* tw, int dir) {
    const int nbf = N / R;
    const int step = N / (Ns * R);
    for (int t = threadIdx.x; t < batch * nbf; t += blockDim.x) {
        const int bidx = t / nbf, j = t - bidx * nbf;
        const cplx<T>* src = in + (size_t)bidx * ld;
        cplx<T>* dst = out + (size_t)bidx * ld;
        const int k = j % Ns;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * nbf];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                cplx<T> w = tw[(r * k * step) % N];
                if (dir > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (R == 2) dft2(v);
        else if (R == 4) dft4(v, dir);
        else if (R == 8) dft8(v, dir);
        else if (R == 3) dft_odd<T, 3>(v, dir);
        else if (R == 5) dft_odd<T, 5>(v, dir);
        else dft_odd<T, 7>(v, dir);
        const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[idxD + r * Ns] = v[r];
    }
}

// Transform `batch` sequences of length N (sequence b at a + b*ld) in place
// semantics: returns the buffer (a or b) holding the result.  dir = -1
// forward (exp(-i ...)), +1 inverse, unnormalised.  Synchronises the block.
template <typename T>
__device__ cplx<T>* fft_batch(cplx<T>* a, cplx<T>* b, int N, int batch, int ld, const cplx<T>* tw, int dir) {
    const FftPlan pl = make_plan(N);
    int Ns = 1;
    cplx<T>* in = a;
    cplx<T>* out = b;
    for (int s = 0; s < pl.ns; ++s) {
        const int R = pl.radix[s];
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

}  // namespace recon
