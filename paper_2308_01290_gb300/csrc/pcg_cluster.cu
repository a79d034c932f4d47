// Z^m step of Algorithm 1 (Sec. II-D), one slice per thread-block cluster.
//
// The normal equations [diag(a^2) + beta~ (dx^T dx + dy^T dy)] z = rhs are
// solved by preconditioned CG with the preconditioner
//   M^-1 = D^-1/2 (mean(a^2) + beta~ L)^-1 D^-1/2,
//   D = diag((a^2 + 4 beta~) / (mean(a^2) + 4 beta~)),
// applied by a 2-D FFT.  A cluster of kClusterCtas CTAs owns one slice for
// the whole solve: CTA c holds a band of R rows for the pointwise and stencil
// work and the row FFTs, and a band of spectrum columns for the column FFTs;
// the row <-> column exchange of the half spectrum goes through distributed
// shared memory.  Dot products are summed per CTA, then over the cluster in
// rank order (identical, deterministic totals in every CTA), so every branch
// on them is uniform over the cluster.  The vectors live in global memory
// (z, r, the two p buffers, y); a slice's working set (~7 MB at 512^2) stays
// in L2 while its cluster iterates.  A persistent grid of clusters takes
// slices from a queue.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "ctx.h"
#include "fft.cuh"
#include "pcg_cluster.h"

namespace cgx = cooperative_groups;

namespace recon {

namespace {

constexpr int kMaxVec = 8;   // float4 vectors of the own row band per thread

struct ClusterArgs {
    const int* slices;        // eligible slice indices
    int n_slices;
    int* queue;               // next index into slices (reset to 0 before launch)
    const SliceGeom* G;
    const SliceConst* C;
    SliceState* S;
    float* z;
    const float* a2;
    const float* rhs;
    float* r;
    float* p0;
    float* p1;
    float* y;
    const cplx<float>* tw;
    const float* sym;
    unsigned long long* acct;
    int smem_x, smem_s;       // complex slots of X (= Y) and S
};

struct Band {
    int nx, ny, pitch, nh, R, r0, r1, c0, c1, nvec;
    long long off;
};

__device__ __forceinline__ Band make_band(const SliceGeom& g, int rank) {
    Band b;
    b.nx = g.nx;
    b.ny = g.ny;
    b.pitch = g.pitch;
    b.nh = g.nh;
    b.off = g.off;
    b.R = 2 * ((g.ny + 2 * kClusterCtas - 1) / (2 * kClusterCtas));
    b.r0 = rank * b.R;
    b.r1 = min(g.ny, b.r0 + b.R);
    if (b.r1 < b.r0) b.r1 = b.r0;
    const int cc = (g.nh + kClusterCtas - 1) / kClusterCtas;
    b.c0 = min(g.nh, rank * cc);
    b.c1 = min(g.nh, b.c0 + cc);
    b.nvec = (b.r1 - b.r0) * (g.nx / 4);
    return b;
}

// Sum NV values over the cluster: block sum, then each CTA adds the 16
// per-CTA totals in rank order.  Every thread returns the same totals.
template <int NV>
__device__ __forceinline__ void cluster_sum(cgx::cluster_group& cl, double (&v)[NV], double* red,
                                            double (*slots)[2][4], int& parity, double* bcast) {
    block_sum<NV>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) (*slots)[parity][q] = v[q];
    }
    cl.sync();
    if (threadIdx.x == 0) {
        double t[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) t[q] = 0.0;
        for (int rk = 0; rk < kClusterCtas; ++rk) {
            double(*rs)[2][4] = cl.map_shared_rank(slots, rk);
#pragma unroll
            for (int q = 0; q < NV; ++q) t[q] += (*rs)[parity][q];
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) bcast[q] = t[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = bcast[q];
    __syncthreads();
    parity ^= 1;
}

__device__ __forceinline__ float4 ld4(const float* p, long long d) { return *reinterpret_cast<const float4*>(p + d); }
__device__ __forceinline__ void st4(float* p, long long d, float4 v) { *reinterpret_cast<float4*>(p + d) = v; }

// 5-point periodic Laplacian of field f at the 4 pixels x0..x0+3 of row yy.
__device__ __forceinline__ float4 lap4(const float* f, const Band& b, int yy, int x0, float4 c) {
    const int yu = yy == 0 ? b.ny - 1 : yy - 1, yd = yy == b.ny - 1 ? 0 : yy + 1;
    const long long row = b.off + (long long)yy * b.pitch;
    const float4 up = ld4(f, b.off + (long long)yu * b.pitch + x0);
    const float4 dn = ld4(f, b.off + (long long)yd * b.pitch + x0);
    const float left = f[row + (x0 == 0 ? b.nx - 1 : x0 - 1)];
    const float right = f[row + (x0 + 4 == b.nx ? 0 : x0 + 4)];
    float4 o;
    o.x = (4.f * c.x - left - c.y) - (up.x + dn.x);
    o.y = (4.f * c.y - c.x - c.z) - (up.y + dn.y);
    o.z = (4.f * c.z - c.y - c.w) - (up.z + dn.z);
    o.w = (4.f * c.w - c.z - right) - (up.w + dn.w);
    return o;
}

__device__ __forceinline__ void vec_pos(const Band& b, int v, int& yy, int& x0) {
    const int per = b.nx / 4;
    const int rr = v / per;
    yy = b.r0 + rr;
    x0 = (v - rr * per) * 4;
}

// Put dsc * value of own-band pixel (yy, x) into the row-FFT buffer X:
// rows r0 + 2b and r0 + 2b + 1 are the real and imaginary parts of sequence b.
__device__ __forceinline__ void put_row(cplx<float>* X, const Band& b, int ld, int yy, int x, float v) {
    const int lr = yy - b.r0;
    float* Xf = reinterpret_cast<float*>(X);
    Xf[2 * ((lr >> 1) * ld + pad8(x)) + (lr & 1)] = v;
}

// A band with an odd number of rows packs its last row with no partner: zero
// the partner (imaginary) inputs so that no stale shared memory enters the FFT.
__device__ __forceinline__ void zero_odd_tail(cplx<float>* X, const Band& b, int ld) {
    const int rows = b.r1 - b.r0;
    if (!(rows & 1)) return;
    float* Xf = reinterpret_cast<float*>(X);
    const int seq = rows >> 1;
    for (int x = threadIdx.x; x < b.nx; x += blockDim.x) Xf[2 * (seq * ld + pad8(x)) + 1] = 0.f;
}

// First half of M^-1: row FFTs of the residual already placed in X (own rows,
// D^-1/2-scaled, two rows per complex sequence) and the split of each packed
// pair into the half spectra of the own rows in S.
__device__ __forceinline__ void rows_to_spectrum(cplx<float>* X, cplx<float>* Y, cplx<float>* Sm,
                                                                 const Band& b, const SliceGeom& g,
                                                                 const cplx<float>* tw) {
    const int ld = padded_len(b.nx);
    const int np = (b.r1 - b.r0 + 1) / 2;
    const cplx<float>* res = X;
    if (np > 0) res = fft_batch<float>(X, Y, b.nx, g.plan_x, np, ld, tw + g.twx, -1);
    // split the packed pairs into half spectra of the own rows
    for (int q = threadIdx.x; q < np * b.nh; q += blockDim.x) {
        const int bb = q / b.nh, k = q - bb * b.nh;
        const cplx<float> zk = res[bb * ld + pad8(k)];
        const cplx<float> zc = res[bb * ld + pad8(k == 0 ? 0 : b.nx - k)];
        const int lr = 2 * bb;
        Sm[lr * b.nh + k] = {0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y)};
        if (b.r0 + lr + 1 < b.r1) Sm[(lr + 1) * b.nh + k] = {0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x)};
    }
}

}  // namespace

__global__ void __launch_bounds__(kClusterThreads, 1) k_pcg_cluster(ClusterArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<float>* X = reinterpret_cast<cplx<float>*>(smem_raw);
    cplx<float>* Y = X + A.smem_x;
    cplx<float>* Sm = Y + A.smem_x;
    __shared__ double red[3 * 32];
    __shared__ double slots[2][4];
    __shared__ double bcast[4];
    __shared__ int s_next;
    __shared__ SliceGeom s_g;
    __shared__ SliceConst s_c;
    cgx::cluster_group cl = cgx::this_cluster();
    const int rank = (int)cl.block_rank();
    int parity = 0;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_next = atomicAdd(A.queue, 1);
        cl.sync();
        const int qi = *cl.map_shared_rank(&s_next, 0);
        cl.sync();   // every CTA has read the index before rank 0 takes the next
        if (qi >= A.n_slices) break;
        const int s = A.slices[qi];
        stage_struct(&s_g, A.G + s);
        stage_struct(&s_c, A.C + s);
        __syncthreads();
        const SliceGeom& g = s_g;
        if (!__ldg(&A.S[s].active)) continue;   // uniform: same state for every CTA
        const Band b = make_band(g, rank);
        const float bt = (float)__ldg(&A.S[s].beta_t);
        const double abar2 = __ldg(&A.S[s].abar2);
        const double bbn = __ldg(&A.S[s].bb);
        const double tol2 = s_c.cg_tol * s_c.cg_tol;
        const float rnum = (float)sqrt(abar2 + 4.0 * (double)bt), b4 = 4.f * bt;
        const int ld = padded_len(b.nx);
        const int ldc = padded_len(b.ny) | 1;
        const cplx<float>* tw = A.tw;

        // ---- r = rhs - A z, rr, and the residual into the row-FFT buffer
        double acc[1] = {0.0};
        zero_odd_tail(X, b, ld);
        {
            float accT = 0.f;
            for (int v = threadIdx.x; v < b.nvec; v += blockDim.x) {
                int yy, x0;
                vec_pos(b, v, yy, x0);
                const long long d = b.off + (long long)yy * b.pitch + x0;
                const float4 zc = ld4(A.z, d), a2 = ld4(A.a2, d), rh = ld4(A.rhs, d);
                const float4 lz = lap4(A.z, b, yy, x0, zc);
                float4 rv;
                rv.x = rh.x - (a2.x * zc.x + bt * lz.x);
                rv.y = rh.y - (a2.y * zc.y + bt * lz.y);
                rv.z = rh.z - (a2.z * zc.z + bt * lz.z);
                rv.w = rh.w - (a2.w * zc.w + bt * lz.w);
                st4(A.r, d, rv);
                accT = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, accT))));
                put_row(X, b, ld, yy, x0 + 0, rv.x * rnum * rsqrtf(a2.x + b4));
                put_row(X, b, ld, yy, x0 + 1, rv.y * rnum * rsqrtf(a2.y + b4));
                put_row(X, b, ld, yy, x0 + 2, rv.z * rnum * rsqrtf(a2.z + b4));
                put_row(X, b, ld, yy, x0 + 3, rv.w * rnum * rsqrtf(a2.w + b4));
            }
            acc[0] = (double)accT;
        }
        __syncthreads();
        rows_to_spectrum(X, Y, Sm, b, g, tw);
        cluster_sum<1>(cl, acc, red, &slots, parity, bcast);   // also: every S band complete
        double rr = acc[0];
        int it = 0;
        bool done = (bbn == 0.0) || !(rr > tol2 * bbn);
        double ry = 0.0, betacg = 0.0;
        int par = 0;
        long long px_iters = 0;
        while (!done) {
            // ---- column pass of M^-1: gather the own columns of all rows
            const int nc = b.c1 - b.c0;
            for (int q = threadIdx.x; q < nc * b.ny; q += blockDim.x) {
                const int yy = q / nc, kk = q - yy * nc;
                const int owner = yy / b.R, lr = yy - owner * b.R;
                const cplx<float>* src = cl.map_shared_rank(Sm, owner);
                X[kk * ldc + pad8(yy)] = src[lr * b.nh + b.c0 + kk];
            }
            cl.sync();   // every band gathered before any scatter overwrites S
            if (nc > 0) {
                cplx<float>* cur = fft_batch<float>(X, Y, b.ny, g.plan_y, nc, ldc, tw + g.twy, -1);
                const float inv_n = (float)(1.0 / ((double)b.nx * (double)b.ny));
                const float* symx = A.sym + g.symx;
                const float* symy = A.sym + g.symy;
                for (int q = threadIdx.x; q < nc * b.ny; q += blockDim.x) {
                    const int kk = q / b.ny, ky = q - kk * b.ny;
                    const float sc = inv_n / ((float)abar2 + bt * (symx[b.c0 + kk] + symy[ky]));
                    cplx<float> v = cur[kk * ldc + pad8(ky)];
                    cur[kk * ldc + pad8(ky)] = {v.x * sc, v.y * sc};
                }
                __syncthreads();
                cur = fft_batch<float>(cur, cur == X ? Y : X, b.ny, g.plan_y, nc, ldc, tw + g.twy, +1);
                for (int q = threadIdx.x; q < nc * b.ny; q += blockDim.x) {
                    const int yy = q / nc, kk = q - yy * nc;
                    const int owner = yy / b.R, lr = yy - owner * b.R;
                    cplx<float>* dst = cl.map_shared_rank(Sm, owner);
                    dst[lr * b.nh + b.c0 + kk] = cur[kk * ldc + pad8(yy)];
                }
            }
            cl.sync();   // every band's solved half spectrum is home
            // ---- inverse row FFTs of the own rows -> y = D^-1/2 (...), r.y
            {
                const int np = (b.r1 - b.r0 + 1) / 2;
                for (int q = threadIdx.x; q < np * b.nx; q += blockDim.x) {
                    const int bb = q / b.nx, n = q - bb * b.nx;
                    const bool herm = n >= b.nh;
                    const int k = herm ? b.nx - n : n;
                    const int lr = 2 * bb;
                    cplx<float> Av = Sm[lr * b.nh + k], Bv = {0.f, 0.f};
                    if (b.r0 + lr + 1 < b.r1) Bv = Sm[(lr + 1) * b.nh + k];
                    if (herm) {
                        Av.y = -Av.y;
                        Bv.y = -Bv.y;
                    }
                    X[bb * ld + pad8(n)] = {Av.x - Bv.y, Av.y + Bv.x};
                }
                __syncthreads();
                const cplx<float>* res = X;
                if (np > 0) res = fft_batch<float>(X, Y, b.nx, g.plan_x, np, ld, tw + g.twx, +1);
                float accT = 0.f;
                for (int q = threadIdx.x; q < np * b.nx; q += blockDim.x) {
                    const int bb = q / b.nx, n = q - bb * b.nx;
                    const cplx<float> v = res[bb * ld + pad8(n)];
                    const int yy = b.r0 + 2 * bb;
                    const long long d0 = b.off + (long long)yy * b.pitch + n;
                    const float y0 = v.x * rnum * rsqrtf(A.a2[d0] + b4);
                    A.y[d0] = y0;
                    accT = fmaf(y0, A.r[d0], accT);
                    if (yy + 1 < b.r1) {
                        const long long d1 = d0 + b.pitch;
                        const float y1 = v.y * rnum * rsqrtf(A.a2[d1] + b4);
                        A.y[d1] = y1;
                        accT = fmaf(y1, A.r[d1], accT);
                    }
                }
                acc[0] = (double)accT;
            }
            cluster_sum<1>(cl, acc, red, &slots, parity, bcast);
            betacg = (it == 0) ? 0.0 : acc[0] / ry;
            ry = acc[0];
            // ---- p = y + beta p_old (own rows)
            float* pold = par ? A.p1 : A.p0;
            float* pnew = par ? A.p0 : A.p1;
            const float bc = (float)betacg;
            for (int v = threadIdx.x; v < b.nvec; v += blockDim.x) {
                int yy, x0;
                vec_pos(b, v, yy, x0);
                const long long d = b.off + (long long)yy * b.pitch + x0;
                float4 pv = ld4(A.y, d);
                if (it > 0) {
                    const float4 po = ld4(pold, d);
                    pv.x = fmaf(bc, po.x, pv.x);
                    pv.y = fmaf(bc, po.y, pv.y);
                    pv.z = fmaf(bc, po.z, pv.z);
                    pv.w = fmaf(bc, po.w, pv.w);
                }
                st4(pnew, d, pv);
            }
            cl.sync();   // p complete for the halo reads
            // ---- q = A p (kept in registers), p.q
            float4 qreg[kMaxVec];
            {
                float accT = 0.f;
#pragma unroll
                for (int k = 0; k < kMaxVec; ++k) {
                    const int v = threadIdx.x + k * blockDim.x;
                    if (v < b.nvec) {
                        int yy, x0;
                        vec_pos(b, v, yy, x0);
                        const long long d = b.off + (long long)yy * b.pitch + x0;
                        const float4 pc = ld4(pnew, d), a2 = ld4(A.a2, d);
                        const float4 lp = lap4(pnew, b, yy, x0, pc);
                        float4 qv;
                        qv.x = a2.x * pc.x + bt * lp.x;
                        qv.y = a2.y * pc.y + bt * lp.y;
                        qv.z = a2.z * pc.z + bt * lp.z;
                        qv.w = a2.w * pc.w + bt * lp.w;
                        qreg[k] = qv;
                        accT = fmaf(pc.x, qv.x, fmaf(pc.y, qv.y, fmaf(pc.z, qv.z, fmaf(pc.w, qv.w, accT))));
                    }
                }
                acc[0] = (double)accT;
            }
            cluster_sum<1>(cl, acc, red, &slots, parity, bcast);
            const double alpha = acc[0] > 0.0 ? ry / acc[0] : 0.0;
            // ---- z += alpha p, r -= alpha q, rr; residual into X for M^-1
            zero_odd_tail(X, b, ld);
            {
                const float al = (float)alpha;
                float accT = 0.f;
#pragma unroll
                for (int k = 0; k < kMaxVec; ++k) {
                    const int v = threadIdx.x + k * blockDim.x;
                    if (v < b.nvec) {
                        int yy, x0;
                        vec_pos(b, v, yy, x0);
                        const long long d = b.off + (long long)yy * b.pitch + x0;
                        float4 zv = ld4(A.z, d), rv = ld4(A.r, d);
                        const float4 pv = ld4(pnew, d), a2 = ld4(A.a2, d);
                        const float4 qv = qreg[k];
                        zv.x = fmaf(al, pv.x, zv.x);
                        zv.y = fmaf(al, pv.y, zv.y);
                        zv.z = fmaf(al, pv.z, zv.z);
                        zv.w = fmaf(al, pv.w, zv.w);
                        rv.x = fmaf(-al, qv.x, rv.x);
                        rv.y = fmaf(-al, qv.y, rv.y);
                        rv.z = fmaf(-al, qv.z, rv.z);
                        rv.w = fmaf(-al, qv.w, rv.w);
                        st4(A.z, d, zv);
                        st4(A.r, d, rv);
                        accT = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, accT))));
                        put_row(X, b, ld, yy, x0 + 0, rv.x * rnum * rsqrtf(a2.x + b4));
                        put_row(X, b, ld, yy, x0 + 1, rv.y * rnum * rsqrtf(a2.y + b4));
                        put_row(X, b, ld, yy, x0 + 2, rv.z * rnum * rsqrtf(a2.z + b4));
                        put_row(X, b, ld, yy, x0 + 3, rv.w * rnum * rsqrtf(a2.w + b4));
                    }
                }
                acc[0] = (double)accT;
            }
            __syncthreads();
            rows_to_spectrum(X, Y, Sm, b, g, tw);
            cluster_sum<1>(cl, acc, red, &slots, parity, bcast);
            rr = acc[0];
            it += 1;
            par ^= 1;
            px_iters += 1;
            done = !(rr > tol2 * bbn) || it >= s_c.cg_max;
        }
        if (rank == 0 && threadIdx.x == 0) {
            SliceState& so = A.S[s];
            so.rr = rr;
            so.cg_it = it;
            so.cg_done = 1;
            // algorithmic bytes: start 16 B/px, each PCG step 56 B/px (see DESIGN)
            const long long npx = (long long)g.nx * g.ny;
            atomicAdd(A.acct + KF_PCG_CLUSTER, (unsigned long long)(npx * 4 * (4 + 14 * px_iters)));
        }
    }
}

namespace {
bool eligible(const SliceGeom& g) {
    if (g.nx % 4 != 0 || g.nx < 32 || g.ny < 32) return false;
    const int R = 2 * ((g.ny + 2 * kClusterCtas - 1) / (2 * kClusterCtas));
    if (R * (g.nx / 4) > kMaxVec * kClusterThreads) return false;
    return true;
}
}  // namespace

int pcg_cluster_setup(Ctx& c) {
    c.cl_slices.clear();
    if (c.precision != 1) return RECON_OK;
    int xs = 0, ss = 0;
    std::vector<int> list;
    for (int s = 0; s < c.n; ++s) {
        const SliceGeom& g = c.sg[s];
        if (!eligible(g)) continue;
        const int R = 2 * ((g.ny + 2 * kClusterCtas - 1) / (2 * kClusterCtas));
        const int cc = (g.nh + kClusterCtas - 1) / kClusterCtas;
        const int x = std::max((R / 2) * padded_len(g.nx), cc * (padded_len(g.ny) | 1));
        const int sm = R * g.nh;
        const size_t bytes = (size_t)(2 * std::max(xs, x) + std::max(ss, sm)) * sizeof(cplx<float>);
        if (bytes > kClusterSmemMax) continue;
        xs = std::max(xs, x);
        ss = std::max(ss, sm);
        list.push_back(s);
    }
    if (!c.use_cluster) list.clear();
    if (list.empty()) return RECON_OK;
    c.cl_smem_x = xs;
    c.cl_smem_s = ss;
    const size_t bytes = (size_t)(2 * xs + ss) * sizeof(cplx<float>);
    RECON_CUDA(cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    RECON_CUDA(cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas, 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_pcg_cluster, &cfg);
    if (e != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return RECON_OK;   // cluster path unavailable: the batched path serves every slice
    }
    c.cl_max_clusters = nclusters;
    c.cl_slices = list;
    void* p = nullptr;
    RECON_CUDA(cudaMalloc(&p, sizeof(int) * (list.size() + 1)));
    c.allocations.push_back(p);
    c.d_cl_slices = static_cast<int*>(p);
    c.d_cl_queue = c.d_cl_slices + list.size();
    RECON_CUDA(cudaMemcpy(c.d_cl_slices, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice));
    c.cl_bytes = bytes;
    for (int s : list) c.sg[s].cluster = 1;
    return RECON_OK;
}

int pcg_cluster_run(Ctx& c) {
    if (c.cl_slices.empty()) return RECON_OK;
    RECON_CUDA(cudaMemsetAsync(c.d_cl_queue, 0, sizeof(int), c.stream));
    ClusterArgs a;
    a.slices = c.d_cl_slices;
    a.n_slices = (int)c.cl_slices.size();
    a.queue = c.d_cl_queue;
    a.G = c.d_geom;
    a.C = c.d_const;
    a.S = c.d_state;
    a.z = static_cast<float*>(c.field[RECON_F_Z]);
    a.a2 = static_cast<const float*>(c.field[RECON_F_A2]);
    a.rhs = static_cast<const float*>(c.field[RECON_F_RHS_Z]);
    a.r = static_cast<float*>(c.field[RECON_F_CG_R]);
    a.p0 = static_cast<float*>(c.field[RECON_F_CG_P0]);
    a.p1 = static_cast<float*>(c.field[RECON_F_CG_P1]);
    a.y = static_cast<float*>(c.field[RECON_F_CG_Y]);
    a.tw = static_cast<const cplx<float>*>(c.d_tw);
    a.sym = static_cast<const float*>(c.d_sym);
    a.acct = c.d_acct;
    a.smem_x = c.cl_smem_x;
    a.smem_s = c.cl_smem_s;
    const int ncl = std::min((int)c.cl_slices.size(), c.cl_max_clusters);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas * ncl, 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = c.cl_bytes;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
        FamTimer t(c, KF_PCG_CLUSTER);
        RECON_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_cluster, a));
    }
    c.launches += 1;
    return RECON_OK;
}

}  // namespace recon
