// Image-quality metrics of Sec. III (PSNR, NMAD, SSIM) of maps against
// reference maps, on the GPU, for batches of slices.
//
// The paper reports the three metrics without printing their definitions;
// the library takes (for each slice, over the pixels of the optional mask,
// all pixels without one):
//   PSNR = 10 log10(peak^2 / MSE), peak = max |ref|;
//   NMAD = sum |x - ref| / sum |ref|;
//   SSIM = mean, over the pixels whose 11 x 11 window lies inside the slice,
//          of ((2 mu_x mu_r + C1)(2 s_xr + C2)) / ((mu_x^2 + mu_r^2 + C1)
//          (s_xx + s_rr + C2)) with the window's normalised Gaussian weights
//          (sigma 1.5), C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = max(ref) -
//          min(ref) over the slice (the mask does not apply to SSIM).
// Sums and window statistics are taken in FP64: a window's variance is a
// small difference of two large moments.  Per-slice sums are reduced in a
// fixed order, so results do not depend on the launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "ctx.h"

namespace recon {
namespace {

constexpr int kIqaThreads = 256;
constexpr int kIqaBlocksPerSlice = 32;
constexpr int kSsimR = 5;                 // window radius (11 x 11)
constexpr int kSsimTile = 16;             // window centres per tile side
constexpr int kSsimIn = kSsimTile + 2 * kSsimR;
constexpr int kSums = 7;                  // see k_iqa_sums

// Block-wide sums of NV doubles in a fixed order; result in thread 0.
template <int NV>
__device__ void block_sum_fixed(double (&v)[NV], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q * 32 + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[q * 32 + w];
            v[q] = s;
        }
    __syncthreads();
}

// Per (slice, block) partials: 0 sum (x - r)^2, 1 sum |x - r|, 2 sum |r|,
// 3 count (all over the mask), 4 max |r| over the mask, 5 min r, 6 max r
// (over the slice).
__global__ void k_iqa_sums(int npx, const float* __restrict__ x, const float* __restrict__ r,
                           const uint8_t* __restrict__ mask, double* part) {
    __shared__ double sh[kSums * 32];
    const int s = blockIdx.y;
    const float* xs = x + (size_t)s * npx;
    const float* rs = r + (size_t)s * npx;
    const uint8_t* ms = mask ? mask + (size_t)s * npx : nullptr;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    double amax = 0.0, rmin = INFINITY, rmax = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += gridDim.x * blockDim.x) {
        const double a = xs[i], b = rs[i];
        rmin = fmin(rmin, b);
        rmax = fmax(rmax, b);
        if (ms && !ms[i]) continue;
        const double d = a - b;
        v[0] += d * d;
        v[1] += fabs(d);
        v[2] += fabs(b);
        v[3] += 1.0;
        amax = fmax(amax, fabs(b));
    }
    block_sum_fixed<4>(v, sh);
    // extrema: warp then block, in a fixed order
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmax(amax, __shfl_down_sync(0xffffffffu, amax, o));
        rmin = fmin(rmin, __shfl_down_sync(0xffffffffu, rmin, o));
        rmax = fmax(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        sh[4 * 32 + warp] = amax;
        sh[5 * 32 + warp] = rmin;
        sh[6 * 32 + warp] = rmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            amax = fmax(amax, sh[4 * 32 + w]);
            rmin = fmin(rmin, sh[5 * 32 + w]);
            rmax = fmax(rmax, sh[6 * 32 + w]);
        }
        double* p = part + ((size_t)s * gridDim.x + blockIdx.x) * kSums;
        p[0] = v[0];
        p[1] = v[1];
        p[2] = v[2];
        p[3] = v[3];
        p[4] = amax;
        p[5] = rmin;
        p[6] = rmax;
    }
}

// Per slice: the partials of k_iqa_sums summed in block order; stats[s] =
// {sse, sad, sar, count, peak, L}.
__global__ void k_iqa_reduce(int nb, const double* part, double* stats) {
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0}, amax = 0.0, rmin = INFINITY, rmax = -INFINITY;
    for (int b = 0; b < nb; ++b) {
        const double* p = part + ((size_t)s * nb + b) * kSums;
        for (int q = 0; q < 4; ++q) v[q] += p[q];
        amax = fmax(amax, p[4]);
        rmin = fmin(rmin, p[5]);
        rmax = fmax(rmax, p[6]);
    }
    double* o = stats + (size_t)s * 6;
    o[0] = v[0];
    o[1] = v[1];
    o[2] = v[2];
    o[3] = v[3];
    o[4] = amax;
    o[5] = rmax - rmin;
}

// SSIM of one 16 x 16 tile of window centres of one slice: the tile and its
// 5-pixel border in shared memory, the five window moments by separable
// Gaussian sums (rows, then columns), the per-pixel SSIM summed over the
// tile.  ssim_part[slice][tile] = that sum.
__global__ void __launch_bounds__(kIqaThreads) k_iqa_ssim(int nx, int ny, const float* __restrict__ x,
                                                          const float* __restrict__ r, const double* stats,
                                                          double* ssim_part) {
    __shared__ float sx[kSsimIn][kSsimIn], sr[kSsimIn][kSsimIn];
    __shared__ double hm[5][kSsimIn][kSsimTile];   // row-filtered x, r, x^2, r^2, x r
    __shared__ double sh[32];
    __shared__ double w[2 * kSsimR + 1];
    const int s = blockIdx.z;
    const int tx = blockIdx.x * kSsimTile, ty = blockIdx.y * kSsimTile;   // first window centre - kSsimR
    const int vx = nx - 2 * kSsimR, vy = ny - 2 * kSsimR;                  // window centres per row / column
    const float* xs = x + (size_t)s * nx * ny;
    const float* rs = r + (size_t)s * nx * ny;
    if (threadIdx.x < 2 * kSsimR + 1) {
        const double t = (double)((int)threadIdx.x - kSsimR);
        w[threadIdx.x] = exp(-t * t / (2.0 * 1.5 * 1.5));
    }
    for (int q = threadIdx.x; q < kSsimIn * kSsimIn; q += blockDim.x) {
        const int ly = q / kSsimIn, lx = q - ly * kSsimIn;
        const int gx = tx + lx, gy = ty + ly;
        const bool in = gx < nx && gy < ny;
        sx[ly][lx] = in ? xs[(size_t)gy * nx + gx] : 0.f;
        sr[ly][lx] = in ? rs[(size_t)gy * nx + gx] : 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i <= 2 * kSsimR; ++i) tot += w[i];
        for (int i = 0; i <= 2 * kSsimR; ++i) w[i] /= tot;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kSsimIn * kSsimTile; q += blockDim.x) {
        const int ly = q / kSsimTile, lx = q - ly * kSsimTile;
        double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i <= 2 * kSsimR; ++i) {
            const double a = sx[ly][lx + i], b = sr[ly][lx + i], wi = w[i];
            m[0] += wi * a;
            m[1] += wi * b;
            m[2] += wi * a * a;
            m[3] += wi * b * b;
            m[4] += wi * a * b;
        }
        for (int k = 0; k < 5; ++k) hm[k][ly][lx] = m[k];
    }
    __syncthreads();
    const double L = stats[(size_t)s * 6 + 5];
    const double c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
    double acc = 0.0;
    for (int q = threadIdx.x; q < kSsimTile * kSsimTile; q += blockDim.x) {
        const int ly = q / kSsimTile, lx = q - ly * kSsimTile;
        if (tx + lx >= vx || ty + ly >= vy) continue;
        double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j <= 2 * kSsimR; ++j)
            for (int k = 0; k < 5; ++k) m[k] += w[j] * hm[k][ly + j][lx];
        const double sxx = m[2] - m[0] * m[0], srr = m[3] - m[1] * m[1], sxr = m[4] - m[0] * m[1];
        acc += ((2.0 * m[0] * m[1] + c1) * (2.0 * sxr + c2)) /
               ((m[0] * m[0] + m[1] * m[1] + c1) * (sxx + srr + c2));
    }
    double v[1] = {acc};
    block_sum_fixed<1>(v, sh);
    if (threadIdx.x == 0) ssim_part[((size_t)s * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = v[0];
}

// out[s] = {PSNR, NMAD, SSIM} of slice s.
__global__ void k_iqa_finish(int n_tiles, int n_valid, const double* stats, const double* ssim_part, double* out) {
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    const double* st = stats + (size_t)s * 6;
    double ss = 0.0;
    for (int t = 0; t < n_tiles; ++t) ss += ssim_part[(size_t)s * n_tiles + t];
    const double mse = st[0] / st[3];
    out[3 * s + 0] = mse > 0.0 ? 10.0 * log10(st[4] * st[4] / mse) : INFINITY;
    out[3 * s + 1] = st[1] / st[2];
    out[3 * s + 2] = ss / (double)n_valid;
}

}  // namespace
}  // namespace recon

using namespace recon;

extern "C" int recon_iqa(int32_t n, int32_t nx, int32_t ny, const float* x, const float* ref, const uint8_t* mask,
                         double* out, void* stream) {
    if (n < 1 || n > 65535 || nx <= 2 * kSsimR || ny <= 2 * kSsimR || nx > RECON_MAX_SIDE || ny > RECON_MAX_SIDE ||
        !x || !ref || !out) {
        set_error("recon_iqa: bad arguments (slices of at least 11 x 11 pixels)");
        return RECON_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const int npx = nx * ny;
    const int tiles_x = (nx - 2 * kSsimR + kSsimTile - 1) / kSsimTile;
    const int tiles_y = (ny - 2 * kSsimR + kSsimTile - 1) / kSsimTile;
    const size_t n_part = (size_t)n * kIqaBlocksPerSlice * kSums, n_stats = (size_t)n * 6;
    const size_t n_ssim = (size_t)n * tiles_x * tiles_y, n_out = (size_t)n * 3;
    double* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, sizeof(double) * (n_part + n_stats + n_ssim + n_out), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    double* part = scratch;
    double* stats = part + n_part;
    double* ssim_part = stats + n_stats;
    double* dout = ssim_part + n_ssim;
    k_iqa_sums<<<dim3(kIqaBlocksPerSlice, n), kIqaThreads, 0, st>>>(npx, x, ref, mask, part);
    k_iqa_reduce<<<n, 32, 0, st>>>(kIqaBlocksPerSlice, part, stats);
    k_iqa_ssim<<<dim3(tiles_x, tiles_y, n), kIqaThreads, 0, st>>>(nx, ny, x, ref, stats, ssim_part);
    k_iqa_finish<<<n, 32, 0, st>>>(tiles_x * tiles_y, (nx - 2 * kSsimR) * (ny - 2 * kSsimR), stats, ssim_part, dout);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * n_out, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "recon_iqa");
    return RECON_OK;
}
