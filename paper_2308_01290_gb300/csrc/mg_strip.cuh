// Fine-level passes of the multigrid-preconditioned Z^m PCG for FP32 slices
// (Alg. 1, Z^m line: [diag(a^2) + beta~ L] z = a b + beta~ div(h, v)),
// written as register-streaming strip kernels.  Included by solver.cu after
// the multigrid tile kernels, whose cycle (Jacobi weight, coarse grids,
// restriction and prolongation) these passes share.
//
// Work layout.  An item is one strip of kStripW = 128 columns (32 lanes of four
// columns, 16-byte accesses) and kStripWarps x rb rows of one slice; warp w of
// the block walks rows y0 + w rb .. y0 + (w + 1) rb - 1 from top to bottom.
// * Horizontal neighbours come from the adjacent lanes by warp shuffles.  The
//   column left of the strip (lane 0) and the column right of its last column
//   (the last active lane) are fetched by those two lanes, with periodic wrap.
// * Vertical neighbours are the rows above and below, kept in registers as the
//   warp walks down the strip.
// * Every row a warp reads arrives through a warp-private ring of
//   kStripDepth shared-memory slots filled by cp.async, so that
//   kStripDepth - 1 rows are in flight while one is computed.  Each lane
//   reads back only its own slot entries: no block barrier is needed until the
//   per-item reduction.
// The slice width must be a multiple of 8 (every lane a whole 16-byte vector;
// at least two active lanes in the last strip of a row).
//
// Per PCG step (rk: residual buffer, par: direction buffer), as in the tile
// kernels but with q = M p no longer stored: k_mgs_fwd forms it again from p
// on a two-pixel halo, and k_mgs_pq forms it only for p.q.  Both call the one
// function m_op, so the two passes compute the same q bit for bit.
//   k_mgs_fwd<UPD>  z += alpha p, r' = r - alpha q (q = M p), r'.r' and the
//                   convergence test; pre-smoothing x1 = w r' / (a^2 + 4 bt)
//                   and the 2x2-mean restriction of r' - M x1 to level 1
//   k_mgs_up<true>  x = w r / (a^2 + 4 bt) + e1 (prolonged), y = x + w (r -
//                   M x) / (a^2 + 4 bt), r.y -> beta_cg
//   k_mgs_pq        p = y + beta_cg p_old, q = M p, p.q -> alpha
// The coarser tile levels l >= 1 whose width is a multiple of 8 run the same
// kernels on their own grid (bt = beta~ / 4^l): k_mgs_fwd<false> is the
// restriction of the level (pre-smoothing from zero, restricted residual),
// k_mgs_up<false> the correction and post-smoothing (no reduction).
#pragma once

namespace recon {

constexpr int kStripW = 128;
constexpr int kStripWarps = 4;
constexpr int kStripThreads = 32 * kStripWarps;
constexpr int kStripDepth = 4;   // ring slots per warp: kStripDepth - 1 rows in flight
constexpr int kStripRowsDefault = 32;

// One lane of a strip item.
struct Lane {
    long long off;   // slice offset in the field pools
    int nx, ny, pitch;
    int x;           // first of the lane's four columns
    int ex;          // this lane's edge column: lane 0 the column left of the strip, the last active lane the
                     // column right of it (periodic)
    int es;          // edge slot: 0 left, 1 right, -1 no edge
    bool act;        // x < nx
};

__device__ __forceinline__ Lane strip_lane(const SliceGeom* G, const Item& it, int lane) {
    const SliceGeom* g = G + it.slice;
    Lane s;
    s.off = __ldg(&g->off);
    s.nx = __ldg(&g->nx);
    s.ny = __ldg(&g->ny);
    s.pitch = __ldg(&g->pitch);
    s.x = it.a + 4 * lane;
    s.act = s.x < s.nx;
    const int w = s.nx - it.a;
    const int last = w >= kStripW ? 31 : w / 4 - 1;   // >= 1 when nx % 8 == 0
    s.es = lane == 0 ? 0 : (lane == last ? 1 : -1);
    s.ex = lane == 0 ? (it.a == 0 ? s.nx - 1 : it.a - 1) : (s.x + 4 == s.nx ? 0 : s.x + 4);
    return s;
}

__device__ __forceinline__ long long strip_row(const Lane& s, int t) {
    return s.off + (long long)wrap_near(t, s.ny) * s.pitch;
}

// Pixels of a strip item (all warps).
__device__ __forceinline__ long long strip_item_px(const Lane& s, const Item& it, int rb) {
    const int h = min(it.b + kStripWarps * rb, s.ny) - it.b;
    return (long long)h * min(kStripW, s.nx - it.a);
}

// The Z^m operator at one pixel, a c + bt ((4c - l - r) - (u + d)): the one
// rounding sequence every strip kernel uses.
__device__ __forceinline__ float m_op(float a, float c, float l, float r, float u, float d, float bt) {
    const float lap = __fsub_rn(__fsub_rn(__fsub_rn(__fmul_rn(4.f, c), l), r), __fadd_rn(u, d));
    return __fmaf_rn(a, c, __fmul_rn(bt, lap));
}
__device__ __forceinline__ float4 m_op4(float4 a, float4 c, float l, float r, float4 u, float4 d, float bt) {
    return make_float4(m_op(a.x, c.x, l, c.y, u.x, d.x, bt), m_op(a.y, c.y, c.x, c.z, u.y, d.y, bt),
                       m_op(a.z, c.z, c.y, c.w, u.z, d.z, bt), m_op(a.w, c.w, c.z, r, u.w, d.w, bt));
}
// Damped Jacobi step from zero: w f / (a + 4 bt).
__device__ __forceinline__ float jac(float f, float a, float b4) {
    return __fdividef(__fmul_rn(mg_omega<float>(), f), __fadd_rn(a, b4));
}
__device__ __forceinline__ float4 jac4(float4 f, float4 a, float b4) {
    return make_float4(jac(f.x, a.x, b4), jac(f.y, a.y, b4), jac(f.z, a.z, b4), jac(f.w, a.w, b4));
}
// Value at the column left of the lane's first column / right of its last.
__device__ __forceinline__ float from_left(const float4& v, float e, const Lane& s) {
    const float l = __shfl_up_sync(0xffffffffu, v.w, 1);
    return s.es == 0 ? e : l;
}
__device__ __forceinline__ float from_right(const float4& v, float e, const Lane& s) {
    const float r = __shfl_down_sync(0xffffffffu, v.x, 1);
    return s.es == 1 ? e : r;
}
__device__ __forceinline__ float4 fma4(float a, float4 b, float4 c) {
    return make_float4(__fmaf_rn(a, b.x, c.x), __fmaf_rn(a, b.y, c.y), __fmaf_rn(a, b.z, c.z),
                       __fmaf_rn(a, b.w, c.w));
}
__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    acc = __fmaf_rn(a.x, b.x, acc);
    acc = __fmaf_rn(a.y, b.y, acc);
    acc = __fmaf_rn(a.z, b.z, acc);
    return __fmaf_rn(a.w, b.w, acc);
}

// Warp-private ring of NF fields: slot k holds one row of each field (the
// lanes' vectors) and the two edge values of the row (slot e[k][f][0] left,
// [1] right; a float2 for fields whose edge is a column pair).
template <int NF>
struct StripRing {
    float4 v[kStripDepth][NF][32];
    float2 e[kStripDepth][NF][2];
};

template <int NF>
constexpr int strip_smem_bytes() {
    return kStripWarps * (int)sizeof(StripRing<NF>);
}

// Streams rows ta .. tb of a warp through its ring: issue(t, slot) starts the
// copies of bundle t, compute(t, slot) runs once they have landed.  The copies
// of bundle t + kStripDepth - 1 go into the slot that bundle t - 1 used, after
// the warp is done with it.
template <typename FI, typename FC>
__device__ __forceinline__ void strip_stream(int ta, int tb, FI issue, FC compute) {
    constexpr int D = kStripDepth;
#pragma unroll
    for (int i = 0; i < D - 1; ++i) {
        if (ta + i <= tb) issue(ta + i, i);
        cp_async_commit();
    }
    int slot = 0;
    for (int t = ta; t <= tb; ++t) {
        __syncwarp();
        const int nt = t + D - 1;
        if (nt <= tb) issue(nt, slot == 0 ? D - 1 : slot - 1);
        cp_async_commit();
        cp_async_wait<D - 1>();
        __syncwarp();
        compute(t, slot);
        slot = slot == D - 1 ? 0 : slot + 1;
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Fine level, start of a PCG step.  UPD: after the update with alpha; else the
// first step (r from k_cg_init, no update).  r is read from rin and, updated,
// written to rout: other items read the old r on their halo in the same launch.
template <bool UPD>
__global__ void __launch_bounds__(kStripThreads, 4) k_mgs_fwd(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                              const SliceConst* C, SliceState* S, Ptrs<float> P,
                                                              int par, const float* rin, float* rout,
                                                              const float* a2, float* F1, int* pending, int rb,
                                                              int lvl) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 p (edge pair), 1 r, 2 a^2 (edge values), 3 z
    StripRing<4>& ring = reinterpret_cast<StripRing<4>*>(strip_dsm)[warp];
    float* z = P.f[RECON_F_Z];
    const float* p = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const Lane s = strip_lane(G, it, lane);
        const SliceGeom* g1p = G1 + it.slice;
        const long long off1 = __ldg(&g1p->off);
        const int pitch1 = __ldg(&g1p->pitch);
        account(P.acct, lvl ? KF_MG_LEVELS : KF_MG_FWD, strip_item_px(s, it, rb) * (UPD ? 25 : 9));
        const float bt = mg_bt<float>(*sp, lvl), b4 = 4.f * bt;
        const float al = UPD ? Sc<float>::alpha(*sp) : 0.f;
        const int r0 = min(it.b + warp * rb, s.ny), r1 = min(r0 + rb, s.ny);
        const int es = s.es < 0 ? 0 : s.es;
        const bool left = s.es == 0;
        float acc = 0.f;
        // the restricted residual of rows (t - 1, t), t odd relative to r0
        auto restrict_store = [&](const float4& e0, const float4& e1, int t) {
            if (!s.act) return;
            const float c0 = __fadd_rn(__fadd_rn(__fadd_rn(e0.x, e0.y), e1.x), e1.y);
            const float c1 = __fadd_rn(__fadd_rn(__fadd_rn(e0.z, e0.w), e1.z), e1.w);
            *reinterpret_cast<float2*>(F1 + off1 + (long long)(t >> 1) * pitch1 + (s.x >> 1)) =
                make_float2(0.25f * c0, 0.25f * c1);
        };
        if (r0 < r1) {
            if constexpr (UPD) {
                // bundle t: p(t) for t in [r0-2, r1+1]; r, a^2 of row t-1 in [r0-1, r1]; z of row t-2 in [r0, r1-1]
                auto issue = [&](int t, int k) {
                    const long long ro = strip_row(s, t);
                    if (s.act) cp_async16(&ring.v[k][0][lane], p + ro + s.x);
                    if (s.es >= 0) cp_async_elem<8>(&ring.e[k][0][es], p + ro + (left ? s.ex - 1 : s.ex));
                    if (t - 1 >= r0 - 1 && t - 1 <= r1) {
                        const long long r1o = strip_row(s, t - 1);
                        if (s.act) {
                            cp_async16(&ring.v[k][1][lane], rin + r1o + s.x);
                            cp_async16(&ring.v[k][2][lane], a2 + r1o + s.x);
                        }
                        if (s.es >= 0) {
                            cp_async_elem<4>(&ring.e[k][1][es], rin + r1o + s.ex);
                            cp_async_elem<4>(&ring.e[k][2][es], a2 + r1o + s.ex);
                        }
                    }
                    if (t - 2 >= r0 && t - 2 < r1 && s.act)
                        cp_async16(&ring.v[k][3][lane], z + strip_row(s, t - 2) + s.x);
                };
                float4 pm2 = {}, pm1 = {};      // p(t-2), p(t-1)
                float2 em2 = {}, em1 = {};      // their edge pairs
                float4 am2 = {};                // a^2(t-2)
                float4 rm2 = {};                // r'(t-2)
                float4 xm3 = {}, xm2 = {};      // x1(t-3), x1(t-2)
                float xe2 = 0.f;                // edge value of x1(t-2)
                float4 res_prev = {};           // residual of the even row of a pair
                auto compute = [&](int t, int k) {
                    const float4 pt = ring.v[k][0][lane];
                    const float2 et = ring.e[k][0][es];
                    if (t >= r0) {
                        // q, r', x1 on row t-1
                        const float4 r_ = ring.v[k][1][lane], a_ = ring.v[k][2][lane];
                        const float re_ = ring.e[k][1][es].x, ae_ = ring.e[k][2][es].x;
                        const float pc_e = left ? em1.y : em1.x;   // p(t-1) at the edge column
                        const float pl = from_left(pm1, pc_e, s), pr = from_right(pm1, pc_e, s);
                        const float4 q = m_op4(a_, pm1, pl, pr, pm2, pt, bt);
                        // q at the edge column: neighbours in the same order as its own lane forms them
                        const float ql = left ? em1.x : pm1.w, qr = left ? pm1.x : em1.y;
                        const float qe = m_op(ae_, pc_e, ql, qr, left ? em2.y : em2.x, left ? et.y : et.x, bt);
                        const float4 rn = fma4(-al, q, r_);
                        const float rne = __fmaf_rn(-al, qe, re_);
                        const float4 x1 = jac4(rn, a_, b4);
                        const float x1e = jac(rne, ae_, b4);
                        if (t >= r0 + 2) {
                            // row t-2: residual, z and r' out, r'.r', restriction
                            const float4 zt = ring.v[k][3][lane];
                            const float xl = from_left(xm2, xe2, s), xr = from_right(xm2, xe2, s);
                            const float4 mx = m_op4(am2, xm2, xl, xr, xm3, x1, bt);
                            const float4 res = make_float4(__fsub_rn(rm2.x, mx.x), __fsub_rn(rm2.y, mx.y),
                                                           __fsub_rn(rm2.z, mx.z), __fsub_rn(rm2.w, mx.w));
                            if (s.act) {
                                const long long ro = strip_row(s, t - 2) + s.x;
                                *reinterpret_cast<float4*>(z + ro) = fma4(al, pm2, zt);
                                *reinterpret_cast<float4*>(rout + ro) = rm2;
                                acc = dot4(rm2, rm2, acc);
                            }
                            if ((t - 2 - r0) & 1) restrict_store(res_prev, res, t - 2);
                            res_prev = res;
                        }
                        xm3 = xm2;
                        xm2 = x1;
                        xe2 = x1e;
                        rm2 = rn;
                        am2 = a_;
                    }
                    pm2 = pm1;
                    em2 = em1;
                    pm1 = pt;
                    em1 = et;
                };
                strip_stream(r0 - 2, r1 + 1, issue, compute);
            } else {
                // bundle t: r, a^2 of row t in [r0-1, r1]
                auto issue = [&](int t, int k) {
                    const long long ro = strip_row(s, t);
                    if (s.act) {
                        cp_async16(&ring.v[k][1][lane], rin + ro + s.x);
                        cp_async16(&ring.v[k][2][lane], a2 + ro + s.x);
                    }
                    if (s.es >= 0) {
                        cp_async_elem<4>(&ring.e[k][1][es], rin + ro + s.ex);
                        cp_async_elem<4>(&ring.e[k][2][es], a2 + ro + s.ex);
                    }
                };
                float4 rm1 = {}, am1 = {}, xm2 = {}, xm1 = {}, res_prev = {};
                float xe1 = 0.f;
                auto compute = [&](int t, int k) {
                    const float4 r_ = ring.v[k][1][lane], a_ = ring.v[k][2][lane];
                    const float4 x1 = jac4(r_, a_, b4);
                    const float x1e = jac(ring.e[k][1][es].x, ring.e[k][2][es].x, b4);
                    if (t >= r0 + 1) {
                        const float xl = from_left(xm1, xe1, s), xr = from_right(xm1, xe1, s);
                        const float4 mx = m_op4(am1, xm1, xl, xr, xm2, x1, bt);
                        const float4 res = make_float4(__fsub_rn(rm1.x, mx.x), __fsub_rn(rm1.y, mx.y),
                                                       __fsub_rn(rm1.z, mx.z), __fsub_rn(rm1.w, mx.w));
                        if ((t - 1 - r0) & 1) restrict_store(res_prev, res, t - 1);
                        res_prev = res;
                    }
                    xm2 = xm1;
                    xm1 = x1;
                    xe1 = x1e;
                    rm1 = r_;
                    am1 = a_;
                };
                strip_stream(r0 - 1, r1, issue, compute);
            }
        }
        if (UPD) {
            const float part[1] = {s.act ? acc : 0.f};
            double a[1];
            block_sum_t<float, 1>(part, a, red);
            double tot[1];
            if (item_reduce<1>(L, w, it.slice, a, tot, red)) {
                SliceState& so = S[it.slice];
                const SliceConst& cs = C[it.slice];
                so.rr = tot[0];
                so.cg_it += 1;
                const bool conv = !(tot[0] > cs.cg_tol * cs.cg_tol * so.bb);
                if (conv || so.cg_it >= cs.cg_max) {
                    so.cg_done = 1;
                    atomicSub(pending, 1);
                }
            }
        }
    }
}

// Correction from level lvl + 1 and post-smoothing on level lvl: FINE (lvl
// 0), y = B r into CG_Y and r.y -> beta_cg; else the level's correction e
// into E (no reduction).  r: residual of the level, a2: its a^2.
template <bool FINE>
__global__ void __launch_bounds__(kStripThreads, 4) k_mgs_up(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                             SliceState* S, Ptrs<float> P, const float* r,
                                                             const float* a2, const float* E1, float* out, int rb,
                                                             int lvl) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 r, 1 a^2 (edge values), 2 e1 (.x, .y of the lane's vector: its two coarse cells; edge value)
    StripRing<3>& ring = reinterpret_cast<StripRing<3>*>(strip_dsm)[warp];
    float* y = out;
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const Lane s = strip_lane(G, it, lane);
        const SliceGeom* g1p = G1 + it.slice;
        const long long off1 = __ldg(&g1p->off);
        const int pitch1 = __ldg(&g1p->pitch);
        account(P.acct, FINE ? KF_MG_Y : KF_MG_LEVELS, strip_item_px(s, it, rb) * 13);
        const float bt = mg_bt<float>(*sp, lvl), b4 = 4.f * bt;
        const int r0 = min(it.b + warp * rb, s.ny), r1 = min(r0 + rb, s.ny);
        const int es = s.es < 0 ? 0 : s.es;
        float acc = 0.f;
        if (r0 < r1) {
            auto issue = [&](int t, int k) {
                const int yy = wrap_near(t, s.ny);
                const long long ro = s.off + (long long)yy * s.pitch;
                const long long co = off1 + (long long)(yy >> 1) * pitch1;
                if (s.act) {
                    cp_async16(&ring.v[k][0][lane], r + ro + s.x);
                    cp_async16(&ring.v[k][1][lane], a2 + ro + s.x);
                    cp_async_elem<8>(&ring.v[k][2][lane], E1 + co + (s.x >> 1));
                }
                if (s.es >= 0) {
                    cp_async_elem<4>(&ring.e[k][0][es], r + ro + s.ex);
                    cp_async_elem<4>(&ring.e[k][1][es], a2 + ro + s.ex);
                    cp_async_elem<4>(&ring.e[k][2][es], E1 + co + (s.ex >> 1));
                }
            };
            float4 rm1 = {}, am1 = {}, xm2 = {}, xm1 = {};
            float xe1 = 0.f;
            auto compute = [&](int t, int k) {
                const float4 r_ = ring.v[k][0][lane], a_ = ring.v[k][1][lane], e_ = ring.v[k][2][lane];
                float4 x = jac4(r_, a_, b4);
                x.x = __fadd_rn(x.x, e_.x);
                x.y = __fadd_rn(x.y, e_.x);
                x.z = __fadd_rn(x.z, e_.y);
                x.w = __fadd_rn(x.w, e_.y);
                const float xe = __fadd_rn(jac(ring.e[k][0][es].x, ring.e[k][1][es].x, b4), ring.e[k][2][es].x);
                if (t >= r0 + 1) {
                    // row t-1: post-smoothing, r.y, y out
                    const float xl = from_left(xm1, xe1, s), xr = from_right(xm1, xe1, s);
                    const float4 mx = m_op4(am1, xm1, xl, xr, xm2, x, bt);
                    float4 yv;
                    yv.x = __fadd_rn(xm1.x, jac(__fsub_rn(rm1.x, mx.x), am1.x, b4));
                    yv.y = __fadd_rn(xm1.y, jac(__fsub_rn(rm1.y, mx.y), am1.y, b4));
                    yv.z = __fadd_rn(xm1.z, jac(__fsub_rn(rm1.z, mx.z), am1.z, b4));
                    yv.w = __fadd_rn(xm1.w, jac(__fsub_rn(rm1.w, mx.w), am1.w, b4));
                    if (s.act) {
                        *reinterpret_cast<float4*>(y + strip_row(s, t - 1) + s.x) = yv;
                        if (FINE) acc = dot4(rm1, yv, acc);
                    }
                }
                xm2 = xm1;
                xm1 = x;
                xe1 = xe;
                rm1 = r_;
                am1 = a_;
            };
            strip_stream(r0 - 1, r1, issue, compute);
        }
        if (FINE) {
            const float part[1] = {acc};
            double a[1];
            block_sum_t<float, 1>(part, a, red);
            double tot[1];
            if (item_reduce<1>(L, w, it.slice, a, tot, red)) {
                SliceState& so = S[it.slice];
                set_betacg(so, (so.cg_it == 0) ? 0.0 : tot[0] / so.ry);
                so.ry = tot[0];
            }
        }
    }
}

// Fine level: p = y + beta_cg p_old (p = y on the first step), q = M p, p.q
// -> alpha.  STOREQ also writes q (the operator test; the PCG does not
// need it).
template <bool STOREQ>
__global__ void __launch_bounds__(kStripThreads, 4) k_mgs_pq(ItemList L, const SliceGeom* G, SliceState* S,
                                                             Ptrs<float> P, int par, int rb) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 y, 1 p_old (edge values), 2 a^2
    StripRing<3>& ring = reinterpret_cast<StripRing<3>*>(strip_dsm)[warp];
    const float* yf = P.f[RECON_F_CG_Y];
    const float* pold = P.f[par ? RECON_F_CG_P1 : RECON_F_CG_P0];
    float* pnew = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    const float* a2 = P.f[RECON_F_A2];
    float* qo = P.f[RECON_F_CG_Q];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const Lane s = strip_lane(G, it, lane);
        const bool first = __ldg(&sp->cg_it) == 0;
        account(P.acct, KF_MG_PQ, strip_item_px(s, it, rb) * (first ? 12 : 16));
        const float bc = first ? 0.f : Sc<float>::betacg(*sp), bt = Sc<float>::beta_t(*sp);
        const int r0 = min(it.b + warp * rb, s.ny), r1 = min(r0 + rb, s.ny);
        const int es = s.es < 0 ? 0 : s.es;
        float acc = 0.f;
        if (r0 < r1) {
            // bundle t: y, p_old of row t in [r0-1, r1]; a^2 of row t-1 in [r0, r1-1]
            auto issue = [&](int t, int k) {
                const long long ro = strip_row(s, t);
                if (s.act) {
                    cp_async16(&ring.v[k][0][lane], yf + ro + s.x);
                    if (!first) cp_async16(&ring.v[k][1][lane], pold + ro + s.x);
                    if (t - 1 >= r0 && t - 1 < r1) cp_async16(&ring.v[k][2][lane], a2 + strip_row(s, t - 1) + s.x);
                }
                if (s.es >= 0) {
                    cp_async_elem<4>(&ring.e[k][0][es], yf + ro + s.ex);
                    if (!first) cp_async_elem<4>(&ring.e[k][1][es], pold + ro + s.ex);
                }
            };
            float4 pm2 = {}, pm1 = {};
            float em1 = 0.f;
            auto compute = [&](int t, int k) {
                float4 pt = ring.v[k][0][lane];
                float et = ring.e[k][0][es].x;
                if (!first) {
                    pt = fma4(bc, ring.v[k][1][lane], pt);
                    et = __fmaf_rn(bc, ring.e[k][1][es].x, et);
                }
                if (t >= r0 && t < r1 && s.act) *reinterpret_cast<float4*>(pnew + strip_row(s, t) + s.x) = pt;
                if (t >= r0 + 1) {
                    // row t-1: q = M p, p.q
                    const float4 a_ = ring.v[k][2][lane];
                    const float pl = from_left(pm1, em1, s), pr = from_right(pm1, em1, s);
                    const float4 q = m_op4(a_, pm1, pl, pr, pm2, pt, bt);
                    if (s.act) {
                        acc = dot4(pm1, q, acc);
                        if (STOREQ) *reinterpret_cast<float4*>(qo + strip_row(s, t - 1) + s.x) = q;
                    }
                }
                pm2 = pm1;
                pm1 = pt;
                em1 = et;
            };
            strip_stream(r0 - 1, r1, issue, compute);
        }
        const float part[1] = {acc};
        double a[1];
        block_sum_t<float, 1>(part, a, red);
        double tot[1];
        if (item_reduce<1>(L, w, it.slice, a, tot, red)) {
            SliceState& so = S[it.slice];
            so.pq = tot[0];
            set_alpha(so, tot[0] > 0.0 ? so.ry / tot[0] : 0.0);
        }
    }
}

}  // namespace recon
