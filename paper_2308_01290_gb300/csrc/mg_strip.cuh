// Fine-level passes of the multigrid-preconditioned Z^m PCG for FP32 slices
// (Alg. 1, Z^m line: [diag(a^2) + beta~ L] z = a b + beta~ div(h, v)),
// written as register-streaming strip kernels.  Included by solver.cu after
// the multigrid tile kernels (the FP64 path), whose grids, restriction and
// prolongation these kernels share.
//
// Work layout.  An item is one strip of kStripW = 128 columns (32 lanes of four
// columns, 16-byte accesses) and kStripWarps x rb rows of one slice; warp w of
// the block walks rows y0 + w rb .. y0 + (w + 1) rb - 1 from top to bottom.
// * Horizontal neighbours come from the adjacent lanes by warp shuffles.  The
//   four columns left of the strip (lane 0) and right of its last column (the
//   last active lane) are fetched by those two lanes as a ghost vector, with
//   periodic wrap; the edge lanes carry the values of the quantities the pass
//   forms on the ghost columns they need (Row::g1..g3, nearest first), with
//   the same rounding sequence as the lane that owns the column.
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
// Smoothing.  The cycle takes two damped Jacobi sweeps (weight w = 0.8,
// J f = w f / (a^2 + 4 bt)) before and after the coarse correction on every
// strip level, as the in-block levels do:
//   pre:  x1 = J f, x2 = x1 + J (f - M x1); restrict f - M x2
//   post: x = x2 + P e, x' = x + J (f - M x), e_out = x' + J (f - M x')
// x2 is formed again in the post-smoothing pass from the same f with the same
// rounding sequence.  Two Jacobi sweeps from zero are a symmetric smoother
// and the post-smoothing is its adjoint, so the cycle stays symmetric positive
// definite as PCG needs.
//
// Per PCG step (rk: residual buffer, par: direction buffer), q = M p is not
// stored: k_mgs_fwd forms it again from p on a three-pixel halo, and k_mgs_pq
// forms it only for p.q.  Both call m_op, so the two passes form the same q
// bit for bit.
//   k_mgs_fwd<true>  z += alpha p, r' = r - alpha q, r'.r' and the
//                    convergence test; pre-smoothing of r' and the 2x2-mean
//                    restriction of r' - M x2 to level 1
//   k_mgs_up<true>   y = B r (correction from level 1, post-smoothing), r.y
//                    -> beta_cg
//   k_mgs_pq         p = y + beta_cg p_old, q = M p, p.q -> alpha
// The coarser tile levels l >= 1 whose width is a multiple of 8 run the same
// kernels on their own grid (bt = beta~ / 4^l): k_mgs_fwd<false> is the
// restriction of a level (pre-smoothing from zero, restricted residual; also
// the fine level's first PCG step), k_mgs_up<false> its correction and
// post-smoothing (no reduction).
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
    int gx;          // first column of this lane's ghost vector: lane 0 the four columns left of the strip, the
                     // last active lane the four right of it (periodic)
    int es;          // ghost slot: 0 left, 1 right, -1 no ghost
    bool act;        // x < nx
    bool left;       // es == 0
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
    s.left = lane == 0;
    s.gx = lane == 0 ? (it.a == 0 ? s.nx - 4 : it.a - 4) : (s.x + 4 == s.nx ? 0 : s.x + 4);
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
// One Jacobi sweep from x: x + J (f - m), m = M x.
__device__ __forceinline__ float sweep(float x, float f, float m, float a, float b4) {
    return __fadd_rn(x, jac(__fsub_rn(f, m), a, b4));
}
// Value at the column left of the lane's first column / right of its last
// (e: the edge lane's nearest ghost value).
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

// A row of one quantity as a lane holds it: its four columns, and in the two
// edge lanes the values on the three ghost columns beyond the strip edge,
// nearest first (other lanes carry unused values there).
struct Row {
    float4 v;
    float g1, g2, g3;
};

// Row from a lane's vector and its ghost vector (left ghost: columns x0-4 ..
// x0-1; right ghost: the four after the strip).
__device__ __forceinline__ Row ld_row(const float4& v, const float4& g, const Lane& s) {
    return Row{v, s.left ? g.w : g.x, s.left ? g.z : g.y, s.left ? g.y : g.z};
}
__device__ __forceinline__ Row jac_row(const Row& f, const Row& a, float b4) {
    return Row{jac4(f.v, a.v, b4), jac(f.g1, a.g1, b4), jac(f.g2, a.g2, b4), jac(f.g3, a.g3, b4)};
}
// M c on a row (u, d: the rows above and below).  On the ghost columns the
// neighbours are taken in the order of the owning lane (left neighbour first),
// so the edge lane forms the owner's value bit for bit; valid one ghost column
// less than c.
__device__ __forceinline__ Row op_row(const Row& a, const Row& c, const Row& u, const Row& d, float bt,
                                      const Lane& s) {
    Row m;
    m.v = m_op4(a.v, c.v, from_left(c.v, c.g1, s), from_right(c.v, c.g1, s), u.v, d.v, bt);
    const float in = s.left ? c.v.x : c.v.w;   // the strip's own column next to the ghost
    m.g1 = m_op(a.g1, c.g1, s.left ? c.g2 : in, s.left ? in : c.g2, u.g1, d.g1, bt);
    m.g2 = m_op(a.g2, c.g2, s.left ? c.g3 : c.g1, s.left ? c.g1 : c.g3, u.g2, d.g2, bt);
    m.g3 = 0.f;
    return m;
}
// x + J (f - m) on a row.
__device__ __forceinline__ Row sweep_row(const Row& x, const Row& f, const Row& m, const Row& a, float b4) {
    Row o;
    o.v = make_float4(sweep(x.v.x, f.v.x, m.v.x, a.v.x, b4), sweep(x.v.y, f.v.y, m.v.y, a.v.y, b4),
                      sweep(x.v.z, f.v.z, m.v.z, a.v.z, b4), sweep(x.v.w, f.v.w, m.v.w, a.v.w, b4));
    o.g1 = sweep(x.g1, f.g1, m.g1, a.g1, b4);
    o.g2 = sweep(x.g2, f.g2, m.g2, a.g2, b4);
    o.g3 = 0.f;
    return o;
}

// Warp-private ring of NF fields: slot k holds one row of each field (the
// lanes' vectors) and the two ghost vectors of the row (g[k][f][0] left,
// [1] right).
template <int NF>
struct StripRing {
    float4 v[kStripDepth][NF][32];
    float4 g[kStripDepth][NF][2];
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

// Copies of one field of row offset ro into ring slot (k, f): the lane's
// vector, and the ghost vector in the edge lanes.
template <int NF>
__device__ __forceinline__ void ring_copy(StripRing<NF>& ring, int k, int f, const float* src, long long ro,
                                          const Lane& s, int lane) {
    if (s.act) cp_async16(&ring.v[k][f][lane], src + ro + s.x);
    if (s.es >= 0) cp_async16(&ring.g[k][f][s.es], src + ro + s.gx);
}
template <int NF>
__device__ __forceinline__ Row ring_row(const StripRing<NF>& ring, int k, int f, const Lane& s, int lane) {
    return ld_row(ring.v[k][f][lane], ring.g[k][f][s.es < 0 ? 0 : s.es], s);
}

// Start of a PCG step on the fine level (UPD: after the update with alpha),
// or the restriction of a coarser tile level lvl (UPD false; also the fine
// level's first step, r from k_cg_init).  The level's residual is read from
// rin; with UPD the updated residual is written to rout (other items read the
// old one on their halo in the same launch).  The pre-smoothed residual,
// restricted as 2x2 means, goes to F1 on grid G1.
template <bool UPD>
__global__ void __launch_bounds__(kStripThreads, 3) k_mgs_fwd(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                              const SliceConst* C, SliceState* S, Ptrs<float> P,
                                                              int par, const float* rin, float* rout,
                                                              const float* a2, float* F1, int* pending, int rb,
                                                              int lvl) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 p, 1 r, 2 a^2, 3 z (lane vectors only)
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
        float acc = 0.f;
        float4 res_prev = {};
        // residual row w (of the restricted pair (w - 1, w) when w - r0 is odd)
        auto restrict_row = [&](const float4& res, int wr) {
            if ((wr - r0) & 1) {
                if (s.act) {
                    const float c0 = __fadd_rn(__fadd_rn(__fadd_rn(res_prev.x, res_prev.y), res.x), res.y);
                    const float c1 = __fadd_rn(__fadd_rn(__fadd_rn(res_prev.z, res_prev.w), res.z), res.w);
                    *reinterpret_cast<float2*>(F1 + off1 + (long long)(wr >> 1) * pitch1 + (s.x >> 1)) =
                        make_float2(0.25f * c0, 0.25f * c1);
                }
            } else {
                res_prev = res;
            }
        };
        auto residual = [&](const Row& f, const Row& m) {
            return make_float4(__fsub_rn(f.v.x, m.v.x), __fsub_rn(f.v.y, m.v.y), __fsub_rn(f.v.z, m.v.z),
                               __fsub_rn(f.v.w, m.v.w));
        };
        if (r0 < r1) {
            Row am1 = {}, am2 = {}, rm1 = {}, rm2 = {}, x1m1 = {}, x1m2 = {}, x2m1 = {}, x2m2 = {};
            if constexpr (UPD) {
                // bundle t: p of row t in [r0-3, r1+2]; r, a^2 of row u = t-1 in [r0-2, r1+1]; z of u in [r0, r1)
                auto issue = [&](int t, int k) {
                    ring_copy(ring, k, 0, p, strip_row(s, t), s, lane);
                    const int u = t - 1;
                    if (u >= r0 - 2 && u <= r1 + 1) {
                        const long long ro = strip_row(s, u);
                        ring_copy(ring, k, 1, rin, ro, s, lane);
                        ring_copy(ring, k, 2, a2, ro, s, lane);
                        if (u >= r0 && u < r1 && s.act) cp_async16(&ring.v[k][3][lane], z + ro + s.x);
                    }
                };
                Row pm2 = {}, pm1 = {};   // p(t-2), p(t-1)
                auto compute = [&](int t, int k) {
                    const Row pt = ring_row(ring, k, 0, s, lane);
                    if (t >= r0 - 1) {
                        // row u = t-1: q = M p, r' = r - alpha q, x1 = J r' (and z += alpha p)
                        const int u = t - 1;
                        const Row au = ring_row(ring, k, 2, s, lane);
                        const Row ru = ring_row(ring, k, 1, s, lane);
                        const Row q = op_row(au, pm1, pm2, pt, bt, s);
                        Row rn;
                        rn.v = fma4(-al, q.v, ru.v);
                        rn.g1 = __fmaf_rn(-al, q.g1, ru.g1);
                        rn.g2 = __fmaf_rn(-al, q.g2, ru.g2);
                        rn.g3 = 0.f;
                        const Row x1 = jac_row(rn, au, b4);
                        if (u >= r0 && u < r1 && s.act)
                            *reinterpret_cast<float4*>(z + strip_row(s, u) + s.x) = fma4(al, pm1.v, ring.v[k][3][lane]);
                        if (t >= r0 + 1) {
                            // row v = t-2: second pre-smoothing sweep
                            const Row x2 = sweep_row(x1m1, rm1, op_row(am1, x1m1, x1m2, x1, bt, s), am1, b4);
                            if (t >= r0 + 3) {
                                // row w = t-3: residual after pre-smoothing, r' out, r'.r', restriction
                                const int wr = t - 3;
                                const float4 res = residual(rm2, op_row(am2, x2m1, x2m2, x2, bt, s));
                                if (s.act) {
                                    *reinterpret_cast<float4*>(rout + strip_row(s, wr) + s.x) = rm2.v;
                                    acc = dot4(rm2.v, rm2.v, acc);
                                }
                                restrict_row(res, wr);
                            }
                            x2m2 = x2m1;
                            x2m1 = x2;
                        }
                        x1m2 = x1m1;
                        x1m1 = x1;
                        rm2 = rm1;
                        rm1 = rn;
                        am2 = am1;
                        am1 = au;
                    }
                    pm2 = pm1;
                    pm1 = pt;
                };
                strip_stream(r0 - 3, r1 + 2, issue, compute);
            } else {
                // bundle t: r, a^2 of row t in [r0-2, r1+1]
                auto issue = [&](int t, int k) {
                    const long long ro = strip_row(s, t);
                    ring_copy(ring, k, 1, rin, ro, s, lane);
                    ring_copy(ring, k, 2, a2, ro, s, lane);
                };
                auto compute = [&](int t, int k) {
                    const Row rt = ring_row(ring, k, 1, s, lane), at = ring_row(ring, k, 2, s, lane);
                    const Row x1 = jac_row(rt, at, b4);
                    if (t >= r0) {
                        // row v = t-1: second pre-smoothing sweep
                        const Row x2 = sweep_row(x1m1, rm1, op_row(am1, x1m1, x1m2, x1, bt, s), am1, b4);
                        if (t >= r0 + 2) {
                            // row w = t-2: residual after pre-smoothing, restriction
                            restrict_row(residual(rm2, op_row(am2, x2m1, x2m2, x2, bt, s)), t - 2);
                        }
                        x2m2 = x2m1;
                        x2m1 = x2;
                    }
                    x1m2 = x1m1;
                    x1m1 = x1;
                    rm2 = rm1;
                    rm1 = rt;
                    am2 = am1;
                    am1 = at;
                };
                strip_stream(r0 - 2, r1 + 1, issue, compute);
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
                    atomicMax(pending + 1, so.cg_it);
                }
            }
        }
    }
}

// Correction from level lvl + 1 and post-smoothing on level lvl: FINE (lvl
// 0), y = B r into `out` (CG_Y) and r.y -> beta_cg; else the level's
// correction into `out` (no reduction).  r: residual of the level, a2: its
// a^2, E1: the correction of level lvl + 1 on grid G1.
template <bool FINE>
__global__ void __launch_bounds__(kStripThreads, 3) k_mgs_up(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                             SliceState* S, Ptrs<float> P, const float* r,
                                                             const float* a2, const float* E1, float* out, int rb,
                                                             int lvl) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 r, 1 a^2, 2 e1 (.x, .y: the lane's two coarse cells; ghost .x: the coarse cell next to the strip)
    StripRing<3>& ring = reinterpret_cast<StripRing<3>*>(strip_dsm)[warp];
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
        // the coarse cell next to the strip: the two ghost columns nearest the strip lie in it
        const int ecx = (s.left ? s.gx + 3 : s.gx) >> 1;
        float acc = 0.f;
        if (r0 < r1) {
            // bundle t: r, a^2 of row t in [r0-3, r1+2]; e1 under row u = t-1 in [r0-2, r1+1]
            auto issue = [&](int t, int k) {
                const long long ro = strip_row(s, t);
                ring_copy(ring, k, 0, r, ro, s, lane);
                ring_copy(ring, k, 1, a2, ro, s, lane);
                const int u = t - 1;
                if (u >= r0 - 2 && u <= r1 + 1) {
                    const long long co = off1 + (long long)(wrap_near(u, s.ny) >> 1) * pitch1;
                    if (s.act) cp_async_elem<8>(&ring.v[k][2][lane], E1 + co + (s.x >> 1));
                    if (s.es >= 0) cp_async_elem<4>(&ring.g[k][2][s.es], E1 + co + ecx);
                }
            };
            Row rm1 = {}, rm2 = {}, rm3 = {}, am1 = {}, am2 = {}, am3 = {};
            Row x1m1 = {}, x1m2 = {}, xm1 = {}, xm2 = {}, xpm1 = {}, xpm2 = {};
            auto compute = [&](int t, int k) {
                const Row rt = ring_row(ring, k, 0, s, lane), at = ring_row(ring, k, 1, s, lane);
                const Row x1 = jac_row(rt, at, b4);
                if (t >= r0 - 1) {
                    // row u = t-1: second pre-smoothing sweep, then the prolonged correction
                    Row x = sweep_row(x1m1, rm1, op_row(am1, x1m1, x1m2, x1, bt, s), am1, b4);
                    const float4 e = ring.v[k][2][lane];
                    const float eg = ring.g[k][2][s.es < 0 ? 0 : s.es].x;
                    x.v.x = __fadd_rn(x.v.x, e.x);
                    x.v.y = __fadd_rn(x.v.y, e.x);
                    x.v.z = __fadd_rn(x.v.z, e.y);
                    x.v.w = __fadd_rn(x.v.w, e.y);
                    x.g1 = __fadd_rn(x.g1, eg);
                    x.g2 = __fadd_rn(x.g2, eg);
                    if (t >= r0 + 1) {
                        // row v = t-2: first post-smoothing sweep
                        const Row xp = sweep_row(xm1, rm2, op_row(am2, xm1, xm2, x, bt, s), am2, b4);
                        if (t >= r0 + 3) {
                            // row w = t-3: second post-smoothing sweep, out (and r.y)
                            const Row y = sweep_row(xpm1, rm3, op_row(am3, xpm1, xpm2, xp, bt, s), am3, b4);
                            if (s.act) {
                                *reinterpret_cast<float4*>(out + strip_row(s, t - 3) + s.x) = y.v;
                                if (FINE) acc = dot4(rm3.v, y.v, acc);
                            }
                        }
                        xpm2 = xpm1;
                        xpm1 = xp;
                    }
                    xm2 = xm1;
                    xm1 = x;
                }
                x1m2 = x1m1;
                x1m1 = x1;
                rm3 = rm2;
                rm2 = rm1;
                rm1 = rt;
                am3 = am2;
                am2 = am1;
                am1 = at;
            };
            strip_stream(r0 - 3, r1 + 2, issue, compute);
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
    // fields: 0 y, 1 p_old, 2 a^2 (lane vectors only)
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
        float acc = 0.f;
        if (r0 < r1) {
            // bundle t: y, p_old of row t in [r0-1, r1]; a^2 of row t-1 in [r0, r1-1]
            auto issue = [&](int t, int k) {
                const long long ro = strip_row(s, t);
                ring_copy(ring, k, 0, yf, ro, s, lane);
                if (!first) ring_copy(ring, k, 1, pold, ro, s, lane);
                if (t - 1 >= r0 && t - 1 < r1 && s.act) cp_async16(&ring.v[k][2][lane], a2 + strip_row(s, t - 1) + s.x);
            };
            Row pm2 = {}, pm1 = {};
            auto compute = [&](int t, int k) {
                Row pt = ring_row(ring, k, 0, s, lane);
                if (!first) {
                    const Row po = ring_row(ring, k, 1, s, lane);
                    pt.v = fma4(bc, po.v, pt.v);
                    pt.g1 = __fmaf_rn(bc, po.g1, pt.g1);
                }
                if (t >= r0 && t < r1 && s.act) *reinterpret_cast<float4*>(pnew + strip_row(s, t) + s.x) = pt.v;
                if (t >= r0 + 1) {
                    // row t-1: q = M p, p.q
                    const float4 a_ = ring.v[k][2][lane];
                    const float4 q = m_op4(a_, pm1.v, from_left(pm1.v, pm1.g1, s), from_right(pm1.v, pm1.g1, s),
                                           pm2.v, pt.v, bt);
                    if (s.act) {
                        acc = dot4(pm1.v, q, acc);
                        if (STOREQ) *reinterpret_cast<float4*>(qo + strip_row(s, t - 1) + s.x) = q;
                    }
                }
                pm2 = pm1;
                pm1 = pt;
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
