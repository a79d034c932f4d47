// Fan-beam input stage: Joseph ray-driven projector A, its exact transpose
// A^T, flat-detector fan-beam FBP, and the synthetic scan used to make test
// and benchmark inputs.
//
// Geometry (shared by all kernels): image pixel (row j, column i) centre
// x = (i - (nx-1)/2) p, y = (j - (ny-1)/2) p; view k at angle
// t = start + arc k / n_views with source sid (cos t, sin t); detector bin b
// at source - sdd (cos t, sin t) + u_b (-sin t, cos t),
// u_b = (b - (n_bins-1)/2) bin_mm.
//
// A: along the dominant axis of the ray the line is sampled once per pixel
// column (row) and linearly interpolated between the two pixels it passes
// between (zero outside the grid); each sample weighs p |r| / |r_dominant|.
// Per-ray set-up is FP64; the marching is FP32 with the fractional index
// evaluated as start + i * slope from FP64-rounded start and slope.
#include <cmath>
#include <mutex>
#include <vector>

#include "ctx.h"

namespace recon {

namespace {

struct RaySetup {
    int xmajor;        // 1: march over columns, 0: over rows
    float f0, df;      // fractional cross index at march index 0 and its slope
    float w;           // step weight
};

__device__ __forceinline__ RaySetup ray_setup(const recon_geometry& g, int view, int bin) {
    const double t = g.start_rad + g.arc_rad * (double)view / (double)g.n_views;
    double s, c;
    sincos(t, &s, &c);
    const double u = ((double)bin - 0.5 * (g.n_bins - 1)) * g.bin_mm;
    const double Sx = g.sid_mm * c, Sy = g.sid_mm * s;
    const double rx = -g.sdd_mm * c - u * s;
    const double ry = -g.sdd_mm * s + u * c;
    const double p = g.pixel_mm;
    const double len = sqrt(rx * rx + ry * ry);
    RaySetup r;
    if (fabs(rx) >= fabs(ry)) {
        r.xmajor = 1;
        // column i: x_i = (i - (nx-1)/2) p; y = Sy + (x_i - Sx) ry/rx; jf = y/p + (ny-1)/2
        const double x0 = -0.5 * (g.nx - 1) * p;
        const double y0 = Sy + (x0 - Sx) * ry / rx;
        r.f0 = (float)(y0 / p + 0.5 * (g.ny - 1));
        r.df = (float)(ry / rx);
        r.w = (float)(p * len / fabs(rx));
    } else {
        r.xmajor = 0;
        const double y0 = -0.5 * (g.ny - 1) * p;
        const double x0 = Sx + (y0 - Sy) * rx / ry;
        r.f0 = (float)(x0 / p + 0.5 * (g.nx - 1));
        r.df = (float)(rx / ry);
        r.w = (float)(p * len / fabs(ry));
    }
    return r;
}

// one thread per ray; sino[(slice * n_views + view) * n_bins + bin]
// Image slice sl at img + sl * stride, rows `pitch` elements apart.
__global__ void k_project(recon_geometry g, int n, const float* __restrict__ img, long long pitch, long long stride,
                          float* __restrict__ sino) {
    const long long nr = (long long)g.n_views * g.n_bins;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= nr * n) return;
    const int sl = (int)(tid / nr);
    const int ray = (int)(tid - (long long)sl * nr);
    const int view = ray / g.n_bins, bin = ray - view * g.n_bins;
    const RaySetup r = ray_setup(g, view, bin);
    const float* im = img + (long long)sl * stride;
    float acc = 0.f;
    if (r.xmajor) {
        for (int i = 0; i < g.nx; ++i) {
            const float jf = fmaf((float)i, r.df, r.f0);
            const float fl = floorf(jf);
            const int j0 = (int)fl;
            const float w1 = jf - fl;
            if (j0 >= 0 && j0 < g.ny) acc += (1.f - w1) * __ldg(im + (long long)j0 * pitch + i);
            if (j0 + 1 >= 0 && j0 + 1 < g.ny) acc += w1 * __ldg(im + (long long)(j0 + 1) * pitch + i);
        }
    } else {
        for (int j = 0; j < g.ny; ++j) {
            const float xf = fmaf((float)j, r.df, r.f0);
            const float fl = floorf(xf);
            const int i0 = (int)fl;
            const float w1 = xf - fl;
            const float* row = im + (long long)j * pitch;
            if (i0 >= 0 && i0 < g.nx) acc += (1.f - w1) * __ldg(row + i0);
            if (i0 + 1 >= 0 && i0 + 1 < g.nx) acc += w1 * __ldg(row + i0 + 1);
        }
    }
    sino[tid] = acc * r.w;
}

// exact transpose of k_project (same samples, scattered with atomics)
// Adds A^T (wt o sino) into img (layout as k_project; wt: per-ray weights
// laid out as sino, or null for none).
__global__ void k_backproject(recon_geometry g, int n, const float* __restrict__ sino, float* img, long long pitch,
                              long long stride, const float* __restrict__ wt) {
    const long long nr = (long long)g.n_views * g.n_bins;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= nr * n) return;
    const int sl = (int)(tid / nr);
    const int ray = (int)(tid - (long long)sl * nr);
    const int view = ray / g.n_bins, bin = ray - view * g.n_bins;
    const RaySetup r = ray_setup(g, view, bin);
    float* im = img + (long long)sl * stride;
    const float v = (wt ? sino[tid] * wt[tid] : sino[tid]) * r.w;
    if (v == 0.f) return;
    if (r.xmajor) {
        for (int i = 0; i < g.nx; ++i) {
            const float jf = fmaf((float)i, r.df, r.f0);
            const float fl = floorf(jf);
            const int j0 = (int)fl;
            const float w1 = jf - fl;
            if (j0 >= 0 && j0 < g.ny) atomicAdd(im + (long long)j0 * pitch + i, (1.f - w1) * v);
            if (j0 + 1 >= 0 && j0 + 1 < g.ny) atomicAdd(im + (long long)(j0 + 1) * pitch + i, w1 * v);
        }
    } else {
        for (int j = 0; j < g.ny; ++j) {
            const float xf = fmaf((float)j, r.df, r.f0);
            const float fl = floorf(xf);
            const int i0 = (int)fl;
            const float w1 = xf - fl;
            float* row = im + (long long)j * pitch;
            if (i0 >= 0 && i0 < g.nx) atomicAdd(row + i0, (1.f - w1) * v);
            if (i0 + 1 >= 0 && i0 + 1 < g.nx) atomicAdd(row + i0 + 1, w1 * v);
        }
    }
}

// FBP step 1: cosine weight sid / sqrt(sid^2 + s^2) (s at the isocentre
// plane) and Ram-Lak ramp h(0) = 1/(4 ds^2), h(odd m) = -1/(pi m ds)^2,
// q(n) = ds sum_k h(n - k) w(k).  One block per (slice, view).  A thread
// forms the two outputs b, b + 1 (b even): the row sits at an odd offset in
// shared memory, so for every odd m the taps b - m, b + 1 - m and b + m,
// b + 1 + m are 8-byte aligned pairs, one vector load each; a warp's pairs are
// consecutive, so the loads are free of bank conflicts.  Each output's sum
// runs over m in increasing order as in a plain loop.
__host__ __device__ inline int fbp_row_pad(int nb) { return nb | 1; }
__host__ __device__ inline int fbp_row_len(int nb) { return 3 * nb + 4; }
__host__ __device__ inline int fbp_filter_smem_floats(int nb) { return fbp_row_len(nb) + (nb + 1) / 2; }

__global__ void k_fbp_filter(recon_geometry g, int n, const float* __restrict__ sino, float* __restrict__ q) {
    extern __shared__ __align__(16) float smem_f[];
    const int nb = g.n_bins;
    const int pad = fbp_row_pad(nb), len = fbp_row_len(nb);
    float* wrow = smem_f;          // weighted row at the odd offset pad, zero-padded
    float* hodd = smem_f + len;    // ds h(m) for odd m = 2t + 1
    const int sv = blockIdx.x;     // slice * n_views + view
    if (sv >= n * g.n_views) return;
    // FP32 throughout: GB300 issues FP64 at a small fraction of its FP32 rate
    const float sid = (float)g.sid_mm;
    const float ds = (float)g.bin_mm * sid / (float)g.sdd_mm;
    const float* src = sino + (long long)sv * nb;
    for (int b = threadIdx.x; b < len; b += blockDim.x) {
        const int k = b - pad;
        float v = 0.f;
        if (k >= 0 && k < nb) {
            const float s = ((float)k - 0.5f * (float)(nb - 1)) * ds;
            v = src[k] * sid / sqrtf(fmaf(s, s, sid * sid));
        }
        wrow[b] = v;
    }
    const float inv_pi2 = (float)(1.0 / (M_PI * M_PI));
    for (int t = threadIdx.x; t < (nb + 1) / 2; t += blockDim.x) {
        const float m = 2.f * (float)t + 1.f;
        hodd[t] = -inv_pi2 / (ds * m * m);   // ds * (-1/(pi m ds)^2)
    }
    __syncthreads();
    const float h0 = 0.25f / ds;   // ds * 1/(4 ds^2)
    for (int b = 2 * threadIdx.x; b < nb; b += 2 * blockDim.x) {
        float acc0 = 0.f, acc1 = 0.f;
        const float* c = wrow + pad + b;   // odd index: c - m and c + m are even for odd m
        // odd offsets m = 2t + 1 on both sides (zero padding outside the row)
        for (int t = 0; 2 * t + 1 < nb; ++t) {
            const int m = 2 * t + 1;
            const float h = hodd[t];
            const float2 lf = *reinterpret_cast<const float2*>(c - m);
            const float2 rt = *reinterpret_cast<const float2*>(c + m);
            acc0 = fmaf(h, lf.x + rt.x, acc0);
            acc1 = fmaf(h, lf.y + rt.y, acc1);
        }
        q[(long long)sv * nb + b] = fmaf(h0, c[0], acc0);
        if (b + 1 < nb) q[(long long)sv * nb + b + 1] = fmaf(h0, c[1], acc1);
    }
}

// The same filter for groups of 8 slices of one geometry, writing the
// group's filtered rows slice-interleaved: q8[(v nb + b) 8 + k] for slice k
// of the group, so that the backprojection reads the 8 slices of a bin as
// two 16-byte loads.  Two blocks per (group, view), one per half of the group
// (slices 4h .. 4h + 3, the 16-byte half h of each bin), filter8_tpr(nb)
// threads per row.  A thread forms 8 consecutive outputs b0 .. b0 + 7 of one
// row and keeps, for each side of the ramp, a window of 16 consecutive
// weighted inputs in registers: four taps move a window by 8, so every four
// taps a thread loads one new group of 8 inputs per side.  The weighted row
// sits in shared memory in 8 phases (element e at (e mod 8) P + e / 8, from
// an offset pad = 1 mod 8), so such a group is 8 loads at fixed offsets from
// one address, and the threads of a warp (consecutive b0 / 8) read
// consecutive words of each phase.  Every output is the same sum in the same
// order as in k_fbp_filter (taps by increasing m, left input plus right).
__host__ __device__ inline int filt8_pad(int nb) { return ((nb + 22) & ~7) + 1; }   // = 1 mod 8, >= nb + 16
__host__ __device__ inline int filt8_phase(int nb) {
    int p = (filt8_pad(nb) + 2 * nb + 40 + 7) / 8;   // the row and the reach of the last windows
    return p + ((4 - p % 32) + 32) % 32;                // = 4 mod 32: conflict-free row fill
}
__host__ __device__ inline int filt8_tpr(int nb) { return ((nb + 7) / 8 + 31) / 32 * 32; }
__host__ __device__ inline int filt8_taps(int nb) { return (nb / 2 + 3) / 4 * 4; }   // ramp taps, padded to 4
__host__ __device__ inline int filt8_smem_floats(int nb) { return filt8_taps(nb) + 32 * filt8_phase(nb); }

// The 8 inputs of group q of a phase-layout row.
__device__ __forceinline__ void filt8_group(const float* ph, int P, int q, float* x) {
#pragma unroll
    for (int p = 0; p < 8; ++p) x[p] = ph[p * P + q];
}

__global__ void __launch_bounds__(512) k_fbp_filter8(recon_geometry g, int n_groups, const float* __restrict__ sino,
                                                     float* __restrict__ q) {
    extern __shared__ __align__(16) float smem_f[];
    const int nb = g.n_bins, nv = g.n_views;
    const int pad = filt8_pad(nb), P = filt8_phase(nb), tpr = filt8_tpr(nb), T = nb / 2;
    const int hl = filt8_taps(nb);
    float* hodd = smem_f;        // ds h(m) for odd m = 2t + 1, zero from t = T
    float* rows = smem_f + hl;   // the half group's 4 weighted rows, 8 P floats each, phase layout
    const int gv = blockIdx.x >> 1, hf = blockIdx.x & 1;   // (group * n_views + view, half)
    if (gv >= n_groups * nv) return;
    const int grp = gv / nv, v = gv - grp * nv;
    const float sid = (float)g.sid_mm;
    const float ds = (float)g.bin_mm * sid / (float)g.sdd_mm;
    const float inv_pi2 = (float)(1.0 / (M_PI * M_PI));
    for (int t = threadIdx.x; t < hl; t += blockDim.x) {
        const float m = 2.f * (float)t + 1.f;
        hodd[t] = t < T ? -inv_pi2 / (ds * m * m) : 0.f;
    }
    const int len = 8 * P;
    for (int qq = threadIdx.x; qq < 4 * len; qq += blockDim.x) {
        const int k = qq / len, e = qq - k * len, kk = e - pad;
        float x = 0.f;
        if (kk >= 0 && kk < nb) {
            const float* src = sino + ((long long)(grp * 8 + 4 * hf + k) * nv + v) * nb;
            const float s = ((float)kk - 0.5f * (float)(nb - 1)) * ds;
            x = src[kk] * sid / sqrtf(fmaf(s, s, sid * sid));
        }
        rows[k * len + (e & 7) * P + (e >> 3)] = x;
    }
    __syncthreads();
    const float h0 = 0.25f / ds;
    const int k = threadIdx.x / tpr, j = threadIdx.x - k * tpr;
    float acc[8];
    const bool on = 8 * j < nb;
    if (on) {
        const float* ph = rows + k * len;
        const int base = pad + 8 * j, Jb = base >> 3;   // base = 8 Jb + 1
        // windows: left inputs 8 (Jb - u - 1) .. 8 (Jb - u) + 7 in (lp, lc), right 8 (Jb + u) .. + 15 in (rc, rn)
        float lp[8], lc[8], rc[8], rn[8];
        filt8_group(ph, P, Jb, lc);
        filt8_group(ph, P, Jb - 1, lp);
        filt8_group(ph, P, Jb, rc);
        filt8_group(ph, P, Jb + 1, rn);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.f;
        const int nblk = T >> 2;
        for (int u = 0; u < nblk; ++u) {
            const float4 h4 = *reinterpret_cast<const float4*>(hodd + 4 * u);
            const float hs[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    // tap t = 4u + s: input b0 + i - m at window offset i - 2s + 8, b0 + i + m at i + 2s + 2
                    const int li = i - 2 * s + 8, ri = i + 2 * s + 2;
                    const float L = li < 8 ? lp[li] : lc[li - 8];
                    const float R = ri < 8 ? rc[ri] : rn[ri - 8];
                    acc[i] = fmaf(hs[s], L + R, acc[i]);
                }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                lc[i] = lp[i];
                rc[i] = rn[i];
            }
            filt8_group(ph, P, Jb - u - 2, lp);
            filt8_group(ph, P, Jb + u + 2, rn);
        }
        auto el = [&](int e) { return ph[(e & 7) * P + (e >> 3)]; };
        for (int t = 4 * nblk; t < T; ++t)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                acc[i] = fmaf(hodd[t], el(base + i - 2 * t - 1) + el(base + i + 2 * t + 1), acc[i]);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = fmaf(h0, el(base + i), acc[i]);
    }
    // out through shared memory (over the rows): slot (k, i, j) at k 8 Q + i Q + j, Q = P
    __syncthreads();
    if (on)
#pragma unroll
        for (int i = 0; i < 8; ++i) rows[k * len + i * P + j] = acc[i];
    __syncthreads();
    float4* q8 = reinterpret_cast<float4*>(q + (long long)grp * 8 * nv * nb);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int o = (b & 7) * P + (b >> 3);
        q8[((long long)v * nb + b) * 2 + hf] = make_float4(rows[o], rows[len + o], rows[2 * len + o], rows[3 * len + o]);
    }
}

// FBP step 2: pixel-driven backprojection of the filtered rows with weight
// 1/U^2, U = (sid - x cos t - y sin t) / sid, detector coordinate at the
// isocentre s' = sid (-x sin t + y cos t) / (U sid), linear interpolation,
// times (arc / n_views) / 2 for a full scan.  A block covers a 16 x (16 R)
// pixel tile of up to S slices (blockIdx.z: the group of slices); each thread
// takes R pixels (16 rows apart) of every slice of its group, so the bin,
// the interpolation weights and 1/U^2 of a (pixel, view) pair are formed
// once for all S slices.  Groups of several slices of one geometry run with
// S = 8, R = 1; single slices with S = 1, R = 2.  Every product that could
// be contracted is written as an explicit FMA or kept apart, so a pixel's
// value is the same in both forms, bit for bit.  The first il_groups groups
// (full groups of 8) come slice-interleaved from k_fbp_filter8, the 8 values
// of a bin in two 16-byte loads; a partial last group comes row by row.
constexpr int kBpTx = 16, kBpTy = 16, kBpGroup = 8;

template <int S, int R>
__global__ void __launch_bounds__(kBpTx * kBpTy, 8)
    k_fbp_backproject(recon_geometry g, int n, const float* __restrict__ q, float* __restrict__ img, int il_groups) {
    // FP32 throughout: GB300 issues FP64 at a small fraction of its FP32 rate
    extern __shared__ float trig[];   // cos, sin per view
    const float a0 = (float)g.start_rad, da = (float)(g.arc_rad / g.n_views);
    for (int v = threadIdx.x + threadIdx.y * kBpTx; v < g.n_views; v += kBpTx * kBpTy) {
        float s, c;
        sincosf(fmaf(da, (float)v, a0), &s, &c);
        trig[2 * v] = c;
        trig[2 * v + 1] = s;
    }
    __syncthreads();
    const int s0 = blockIdx.z * S;
    const int ns = n - s0 < S ? n - s0 : S;
    const int i = blockIdx.x * kBpTx + threadIdx.x;
    const int j0 = blockIdx.y * (kBpTy * R) + threadIdx.y;
    const float sid = (float)g.sid_mm;
    const float inv_ds = (float)g.sdd_mm / ((float)g.bin_mm * sid);
    const float bc = 0.5f * (g.n_bins - 1);
    const float pix = (float)g.pixel_mm;
    const float x = fmaf(-0.5f, (float)(g.nx - 1), (float)i) * pix;
    float y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) y[r] = fmaf(-0.5f, (float)(g.ny - 1), (float)(j0 + r * kBpTy)) * pix;
    const long long sstride = (long long)g.n_views * g.n_bins;
    const float* qs = q + s0 * sstride;   // a full group's interleaved rows start there too
    const bool il = S == 8 && (int)blockIdx.z < il_groups;
    const float kb = sid * inv_ds;
    const unsigned nb = (unsigned)g.n_bins;
    float acc[R][S];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < S; ++k) acc[r][k] = 0.f;
    for (int v = 0; v < g.n_views; ++v) {
        const float c = trig[2 * v], s = trig[2 * v + 1];
        const float xc = x * c, xs = x * s;
        const float* row = qs + (long long)v * g.n_bins;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float L = sid - fmaf(y[r], s, xc);
            const float invL = __fdividef(1.f, L);
            const float bf = fmaf(fmaf(y[r], c, -xs) * kb, invL, bc);
            const float fl = floorf(bf);
            const int b0 = (int)fl;
            const float w1 = bf - fl;
            // 1/U^2 = (sid / L)^2, sid^2 applied after the sum; bins off the
            // detector take weight 0 (and read bin 0)
            const float u2 = invL * invL;
            const float w0 = 1.f - w1;
            const bool in0 = (unsigned)b0 < nb, in1 = (unsigned)(b0 + 1) < nb;
            const float e0 = in0 ? w0 * u2 : 0.f, e1 = in1 ? w1 * u2 : 0.f;
            const int o0 = in0 ? b0 : 0, o1 = in1 ? b0 + 1 : 0;
            if constexpr (S == 8) {
                if (il) {
                    // the 8 slices of bin o: two 16-byte loads
                    const float4* r4 = reinterpret_cast<const float4*>(qs + (long long)v * g.n_bins * 8);
                    const float4 a0 = __ldg(r4 + 2 * o0), a1 = __ldg(r4 + 2 * o0 + 1);
                    const float4 c0 = __ldg(r4 + 2 * o1), c1 = __ldg(r4 + 2 * o1 + 1);
                    const float qa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float qb[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                    for (int k = 0; k < 8; ++k) acc[r][k] = fmaf(e0, qa[k], fmaf(e1, qb[k], acc[r][k]));
                    continue;
                }
            }
#pragma unroll
            for (int k = 0; k < S; ++k)
                if (k < ns) {
                    const float* rk = row + k * sstride;
                    acc[r][k] = fmaf(e0, __ldg(rk + o0), fmaf(e1, __ldg(rk + o1), acc[r][k]));
                }
        }
    }
    if (i >= g.nx) return;
    const float scale = 0.5f * da * sid * sid;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = j0 + r * kBpTy;
        if (j >= g.ny) continue;
#pragma unroll
        for (int k = 0; k < S; ++k)
            if (k < ns) img[(long long)(s0 + k) * g.nx * g.ny + (long long)j * g.nx + i] = acc[r][k] * scale;
    }
}

// rho_e z with z = (Z / Z_w)^m (the photoelectric line-integral map)
__global__ void k_rho_z(long long npx, const float* Z, const float* rho, float* out, float zw, float m) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    out[i] = rho[i] * powf(Z[i] / zw, m);
}

// expected counts I0 sum_b w_b exp(-S (P_b A1 + KN_b A2)), Gaussian noise,
// floor 0.5, -log(counts / I0)
__global__ void k_counts(long long nrays, const float* A1, const float* A2, const double* tab, int nb_lo, int nb_hi,
                         const float* noise, double i0, double S, float* lo, float* hi) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrays) return;
    const double a1 = A1[i], a2 = A2[i];
    for (int arm = 0; arm < 2; ++arm) {
        const int nb = arm ? nb_hi : nb_lo;
        const double* t = tab + (arm ? 3 * nb_lo : 0);
        double lam = 0.0;
        for (int b = 0; b < nb; ++b) lam += t[3 * b] * exp(-S * (t[3 * b + 1] * a1 + t[3 * b + 2] * a2));
        lam *= i0;
        double cnt = lam;
        if (noise) cnt = lam + sqrt(lam) * (double)noise[arm * nrays + i];
        cnt = cnt < 0.5 ? 0.5 : cnt;
        (arm ? hi : lo)[i] = (float)(-log(cnt / i0));
    }
}

int check_geom(const recon_geometry& g) {
    if (g.nx < 1 || g.ny < 1 || g.nx > RECON_MAX_SIDE || g.ny > RECON_MAX_SIDE || g.n_views < 1 || g.n_bins < 1 ||
        !(g.pixel_mm > 0) || !(g.sid_mm > 0) || !(g.sdd_mm > g.sid_mm) || !(g.bin_mm > 0)) {
        set_error("invalid fan-beam geometry");
        return RECON_EINVAL;
    }
    const double half_diag = 0.5 * g.pixel_mm * std::sqrt((double)g.nx * g.nx + (double)g.ny * g.ny);
    if (half_diag >= g.sid_mm) {
        set_error("image reaches the source circle");
        return RECON_EINVAL;
    }
    return RECON_OK;
}

}  // namespace

int ct_project(const recon_geometry& g, int n, const float* img, float* sino, cudaStream_t st, long long* launches) {
    int rc = check_geom(g);
    if (rc) return rc;
    return ct_project_pitched(g, n, img, g.nx, (long long)g.nx * g.ny, sino, st, launches);
}

int ct_project_pitched(const recon_geometry& g, int n, const float* img, long long pitch, long long stride,
                       float* sino, cudaStream_t st, long long* launches) {
    const long long total = (long long)n * g.n_views * g.n_bins;
    if (total <= 0) return RECON_OK;
    k_project<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g, n, img, pitch, stride, sino);
    if (launches) *launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

int ct_backproject_add(const recon_geometry& g, int n, const float* sino, float* img, long long pitch,
                       long long stride, cudaStream_t st, long long* launches, const float* wt) {
    const long long total = (long long)n * g.n_views * g.n_bins;
    if (total <= 0) return RECON_OK;
    k_backproject<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g, n, sino, img, pitch, stride, wt);
    if (launches) *launches += 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

int ct_backproject(const recon_geometry& g, int n, const float* sino, float* img, cudaStream_t st,
                   long long* launches) {
    int rc = check_geom(g);
    if (rc) return rc;
    RECON_CUDA(cudaMemsetAsync(img, 0, sizeof(float) * (size_t)n * g.nx * g.ny, st));
    return ct_backproject_add(g, n, sino, img, g.nx, (long long)g.nx * g.ny, st, launches);
}

int ct_fbp_check(const recon_geometry& g, int n) {
    if (int rc = check_geom(g)) return rc;
    // the filter keeps one weighted row and the odd ramp taps in shared
    // memory, the backprojection the trigonometry of every view
    if ((size_t)g.n_views * 2 * sizeof(float) > 48 * 1024 ||
        (size_t)fbp_filter_smem_floats(g.n_bins) * sizeof(float) > 48 * 1024 || n < 1 || n > 65535 ||
        (long long)n * g.n_views > 0x7fffffffLL) {
        set_error("FBP: too many views or bins for the shared-memory tables, or too many slices");
        return RECON_EINVAL;
    }
    return RECON_OK;
}

int ct_fbp(const recon_geometry& g, int n, const float* sino, float* img, float* scratch, cudaStream_t st,
           long long* launches) {
    if (int rc = ct_fbp_check(g, n)) return rc;
    const size_t fsm = fbp_filter_smem_floats(g.n_bins) * sizeof(float);
    const size_t fsm8 = filt8_smem_floats(g.n_bins) * sizeof(float);
    // full groups of 8 slices: filtered slice-interleaved (where the 4 rows of a half group fit 48 KB of shared
    // memory, up to about 880 bins); the rest row by row
    const int il_groups = (n >= 8 && fsm8 <= 48 * 1024) ? n / kBpGroup : 0;
    const long long sstride = (long long)g.n_views * g.n_bins;
    int k = 0;
    if (il_groups > 0) {
        k_fbp_filter8<<<2 * il_groups * g.n_views, 4 * filt8_tpr(g.n_bins), fsm8, st>>>(g, il_groups, sino, scratch);
        ++k;
    }
    const int rest = n - kBpGroup * il_groups;
    if (rest > 0) {
        const long long o = (long long)kBpGroup * il_groups * sstride;
        k_fbp_filter<<<rest * g.n_views, 256, fsm, st>>>(g, rest, sino + o, scratch + o);
        ++k;
    }
    const size_t trig_bytes = 2 * g.n_views * sizeof(float);
    if (n >= 2) {
        const dim3 grid((g.nx + kBpTx - 1) / kBpTx, (g.ny + kBpTy - 1) / kBpTy, (n + kBpGroup - 1) / kBpGroup);
        k_fbp_backproject<kBpGroup, 1><<<grid, dim3(kBpTx, kBpTy), trig_bytes, st>>>(g, n, scratch, img, il_groups);
    } else {
        const dim3 grid((g.nx + kBpTx - 1) / kBpTx, (g.ny + 2 * kBpTy - 1) / (2 * kBpTy), n);
        k_fbp_backproject<1, 2><<<grid, dim3(kBpTx, kBpTy), trig_bytes, st>>>(g, n, scratch, img, 0);
    }
    if (launches) *launches += k + 1;
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

}  // namespace recon

using namespace recon;

extern "C" int recon_project(const recon_geometry* geom, int32_t n, const float* img, float* sino, void* stream) {
    if (!geom || n < 1 || !img || !sino) {
        set_error("recon_project: bad arguments");
        return RECON_EINVAL;
    }
    return ct_project(*geom, n, img, sino, (cudaStream_t)stream, nullptr);
}

extern "C" int recon_backproject(const recon_geometry* geom, int32_t n, const float* sino, float* img, void* stream) {
    if (!geom || n < 1 || !img || !sino) {
        set_error("recon_backproject: bad arguments");
        return RECON_EINVAL;
    }
    return ct_backproject(*geom, n, sino, img, (cudaStream_t)stream, nullptr);
}

extern "C" int recon_fbp(const recon_geometry* geom, int32_t n, const float* sino, float* img, void* stream) {
    if (!geom || n < 1 || !img || !sino) {
        set_error("recon_fbp: bad arguments");
        return RECON_EINVAL;
    }
    // arguments are checked before any device call or allocation
    if (int rc = ct_fbp_check(*geom, n)) return rc;
    float* scratch = nullptr;
    const size_t bytes = sizeof(float) * (size_t)n * geom->n_views * geom->n_bins;
    cudaError_t e = cudaMallocAsync((void**)&scratch, bytes, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    int rc = ct_fbp(*geom, n, sino, img, scratch, (cudaStream_t)stream, nullptr);
    cudaFreeAsync(scratch, (cudaStream_t)stream);
    return rc;
}

// Scratch of recon_fbp_noalloc: the filtered sinograms of one call.  In host
// code this name stands for the symbol, not a device address; the address is
// looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) float g_fbp_noalloc_scratch[RECON_FBP_NOALLOC_MAX];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

extern "C" int recon_fbp_noalloc(const recon_geometry* geom, int32_t n, const float* sino, float* img, void* stream) {
    if (!geom || n < 1 || !img || !sino) {
        set_error("recon_fbp_noalloc: bad arguments");
        return RECON_EINVAL;
    }
    if (int rc = ct_fbp_check(*geom, n)) return rc;
    const long long need = (long long)n * geom->n_views * geom->n_bins;
    if (need > (long long)RECON_FBP_NOALLOC_MAX) {
        set_error("recon_fbp_noalloc: n * n_views * n_bins exceeds RECON_FBP_NOALLOC_MAX floats of scratch");
        return RECON_EINVAL;
    }
    int dev = 0;
    RECON_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("recon_fbp_noalloc: device index out of range");
        return RECON_EINVAL;
    }
    float* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            RECON_CUDA(cudaGetSymbolAddress(&p, g_fbp_noalloc_scratch));
            g_noalloc_ptr[dev] = static_cast<float*>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    return ct_fbp(*geom, n, sino, img, scratch, (cudaStream_t)stream, nullptr);
}

extern "C" int recon_simulate(const recon_geometry* geom, const recon_params* params, int32_t n, const float* Z,
                              const float* rhoe, const float* noise, double i0, float* sino_low, float* sino_high,
                              void* stream) {
    if (!geom || !params || n < 1 || !Z || !rhoe || !sino_low || !sino_high || !(i0 > 0)) {
        set_error("recon_simulate: bad arguments");
        return RECON_EINVAL;
    }
    if (int rc = check_geom(*geom)) return rc;
    const cudaStream_t st = (cudaStream_t)stream;
    const long long npx = (long long)n * geom->nx * geom->ny;
    const long long nrays = (long long)n * geom->n_views * geom->n_bins;
    // per-bin table (weight, P(E_b), KN(E_b)) of both arms
    std::vector<double> e, w, tab;
    int nbs[2];
    const recon_spectrum* arms[2] = {&params->low, &params->high};
    for (int a = 0; a < 2; ++a) {
        spectrum_bins(*arms[a], e, w);
        nbs[a] = (int)e.size();
        for (size_t b = 0; b < e.size(); ++b) {
            tab.push_back(w[b]);
            tab.push_back(photo_per_z(e[b]));
            tab.push_back(klein_nishina_barn(e[b]));
        }
    }
    float *rz = nullptr, *A1 = nullptr, *A2 = nullptr;
    double* dtab = nullptr;
    // on any failure the buffers already taken are released below
    cudaError_t err = cudaMallocAsync((void**)&rz, sizeof(float) * npx, st);
    if (err == cudaSuccess) err = cudaMallocAsync((void**)&A1, sizeof(float) * nrays, st);
    if (err == cudaSuccess) err = cudaMallocAsync((void**)&A2, sizeof(float) * nrays, st);
    if (err == cudaSuccess) err = cudaMallocAsync((void**)&dtab, sizeof(double) * tab.size(), st);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(dtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) {
        k_rho_z<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(npx, Z, rhoe, rz, (float)water_z(),
                                                               (float)z_exponent());
        err = cudaGetLastError();
    }
    int rc = err == cudaSuccess ? RECON_OK : cuda_fail(err, "recon_simulate");
    if (!rc) rc = ct_project(*geom, n, rz, A1, st, nullptr);
    if (!rc) rc = ct_project(*geom, n, rhoe, A2, st, nullptr);
    if (!rc) {
        k_counts<<<(unsigned)((nrays + 255) / 256), 256, 0, st>>>(nrays, A1, A2, dtab, nbs[0], nbs[1], noise, i0,
                                                                  scale_per_mm(), sino_low, sino_high);
        err = cudaGetLastError();
        if (err != cudaSuccess) rc = cuda_fail(err, "k_counts");
    }
    // the host table must outlive the async copy
    cudaStreamSynchronize(st);
    if (rz) cudaFreeAsync(rz, st);
    if (A1) cudaFreeAsync(A1, st);
    if (A2) cudaFreeAsync(A2, st);
    if (dtab) cudaFreeAsync(dtab, st);
    return rc;
}
