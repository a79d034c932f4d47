// Fine-level passes of the multigrid-preconditioned Z^m PCG for FP32 slices
// up to kBandMaxW columns wide (Alg. 1, Z^m line), as register-streaming band
// kernels: the strip kernels' arithmetic (mg_strip.cuh: same rounding
// sequence, same smoothing, same fusion of q = M p into the update pass, so
// every value is the strip kernels' bit for bit) without ghost columns.
// Included by solver.cu after mg_strip.cuh.
//
// Work layout.  A row of a level nx columns wide is covered by G = nx / 128
// (rounded up) warps of one block, lanes of four columns (16-byte accesses).
// Those G warps walk one band of rb rows together from top to bottom; a block
// of kStripWarps warps holds 4 / G such groups (one when G = 3: the fourth
// warp idles), so an item is 4 / G bands of one slice stacked vertically.
// * Horizontal neighbours come from the adjacent lanes by warp shuffles.  Each
//   warp's first column and last (active) column are published in shared
//   memory, and after a barrier of the group the two edge lanes take their
//   outer neighbour from there: the chunk to the left (the last chunk for the
//   first column) and the chunk to the right (the first chunk for column
//   nx - 1).  The whole row sits in one group, so the periodic boundary
//   (reading R6) needs no ghost columns, and every quantity is formed once per
//   column: no lane carries another lane's values.
// * A pass forms its stencils on rows that lag one step behind each other
//   (q on row t-1 from p, the next sweep on row t-2 from the first, ...), so
//   every stencil of a step takes neighbours of values formed in the step
//   before.  Those are exchanged together at the end of each step: one barrier
//   per row, and the stencils of a step are independent of each other.
// * Vertical neighbours and the cp.async row rings are as in the strip
//   kernels: a warp-private ring of kStripDepth slots per field.
// The edge values alternate between two shared-memory buffers: between two
// uses of one buffer every warp of the group passes the barrier of the other,
// so no warp overwrites an edge that another has still to read.
#pragma once

namespace recon {

constexpr int kBandMaxW = kStripWarps * kStripW;   // widest level the band kernels take (512)

// Warps per row (G) of a level nx columns wide, and row bands per item.
__host__ __device__ __forceinline__ int band_warps(int nx) { return (nx + kStripW - 1) / kStripW; }
__host__ __device__ __forceinline__ int band_groups(int nx) {
    const int g = band_warps(nx);
    return g == 3 ? 1 : kStripWarps / g;
}

// One lane of a band item.
struct BandLane {
    long long off;
    int nx, ny, pitch;
    int x;       // first of the lane's four columns
    int G;       // warps per row
    int grp;     // the warp's row band within the item (>= band_groups: idle warp)
    int wg;      // the warp's chunk of the row (columns wg * 128 ..)
    int lastw;   // last lane of this warp holding columns
    int lsrc;    // chunk whose last column lies left of column wg * 128
    int rsrc;    // chunk whose first column lies right of the warp's last column
    bool act;    // x < nx
    bool idle;
};

__device__ __forceinline__ BandLane band_lane(const SliceGeom* G, int lane, int warp, int slice) {
    const SliceGeom* g = G + slice;
    BandLane b;
    b.off = __ldg(&g->off);
    b.nx = __ldg(&g->nx);
    b.ny = __ldg(&g->ny);
    b.pitch = __ldg(&g->pitch);
    b.G = band_warps(b.nx);
    b.grp = warp / b.G;
    b.wg = warp - b.grp * b.G;
    b.idle = b.grp >= band_groups(b.nx);
    b.x = b.wg * kStripW + 4 * lane;
    b.act = b.x < b.nx;
    const int w = b.nx - b.wg * kStripW;   // columns from this chunk on (>= 8: widths are multiples of 8)
    b.lastw = w >= kStripW ? 31 : w / 4 - 1;
    b.lsrc = b.wg == 0 ? b.G - 1 : b.wg - 1;
    b.rsrc = b.wg == b.G - 1 ? 0 : b.wg + 1;
    return b;
}

__device__ __forceinline__ long long band_row(const BandLane& b, int t) {
    return b.off + (long long)wrap_near(t, b.ny) * b.pitch;
}

// Pixels of a band item (all groups).
__device__ __forceinline__ long long band_item_px(const BandLane& b, const Item& it, int rb) {
    const int h = min(it.b + band_groups(b.nx) * rb, b.ny) - it.b;
    return (long long)h * b.nx;
}

// Barrier of row-band group grp (named barriers 1 .. kStripWarps; immediate
// ids, so that the kernels reserve only those).
__device__ __forceinline__ void band_bar(int grp, int count) {
    switch (grp) {
        case 0: asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory"); break;
        case 1: asm volatile("bar.sync 2, %0;" ::"r"(count) : "memory"); break;
        case 2: asm volatile("bar.sync 3, %0;" ::"r"(count) : "memory"); break;
        default: asm volatile("bar.sync 4, %0;" ::"r"(count) : "memory"); break;
    }
}

// Edge values of up to four quantities of one item: [buffer][group][chunk]
// [0: the chunk's first column, 1: its last column].
struct BandEdges4 {
    float4 e[2][kStripWarps][kStripWarps][2];
};

__device__ __forceinline__ float f4_get(const float4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Left and right neighbours (lr[k].x: column x - 1, lr[k].y: column x + 4) of
// the lane's four columns of each of c[0 .. N-1], through one barrier of the
// band's warps.  Every warp of the band calls it at the same point of its walk.
template <int N>
__device__ __forceinline__ void band_xchg(const float4 (&c)[N], const BandLane& b, int lane, BandEdges4& E,
                                          int& buf, float2 (&lr)[N]) {
    static_assert(N >= 1 && N <= 4, "up to four quantities");
    float4(&e)[kStripWarps][2] = E.e[buf][b.grp];
    float fv[4] = {0.f, 0.f, 0.f, 0.f}, lv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < N; ++k) {
        fv[k] = c[k].x;
        lv[k] = c[k].w;
    }
    if (lane == 0) e[b.wg][0] = make_float4(fv[0], fv[1], fv[2], fv[3]);
    if (lane == b.lastw) e[b.wg][1] = make_float4(lv[0], lv[1], lv[2], lv[3]);
    band_bar(b.grp, 32 * b.G);
    const float4 Lv = e[b.lsrc][1], Rv = e[b.rsrc][0];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float up = __shfl_up_sync(0xffffffffu, c[k].w, 1);
        const float dn = __shfl_down_sync(0xffffffffu, c[k].x, 1);
        lr[k] = make_float2(lane == 0 ? f4_get(Lv, k) : up, lane == b.lastw ? f4_get(Rv, k) : dn);
    }
    buf ^= 1;
}

__device__ __forceinline__ float4 sweep4(const float4& x, const float4& f, const float4& m, const float4& a, float b4) {
    return make_float4(sweep(x.x, f.x, m.x, a.x, b4), sweep(x.y, f.y, m.y, a.y, b4), sweep(x.z, f.z, m.z, a.z, b4),
                       sweep(x.w, f.w, m.w, a.w, b4));
}

template <int NF>
struct BandRing {
    float4 v[kStripDepth][NF][32];
};

template <int NF>
constexpr int band_smem_bytes() {
    return kStripWarps * (int)sizeof(BandRing<NF>);
}

template <int K>
using Slot = std::integral_constant<int, K>;
using Full = std::true_type;
using Edge = std::false_type;

// Streams rows ta .. tb of a warp through its ring as strip_stream does, with
// compute(t, slot, full).  Rows sa .. sb are the steady part of the walk,
// where every condition of compute on t holds: there the rows go four at a
// time with the ring slots and `full` as compile-time constants, so compute
// drops its tests and indexes the ring with immediate offsets.  Elsewhere
// slot is a run-time int and full is false.
template <typename FI, typename FC>
__device__ __forceinline__ void band_stream(int ta, int tb, int sa, int sb, FI issue, FC compute) {
    constexpr int D = kStripDepth;
    static_assert(D == 4, "four rows per steady round");
#pragma unroll
    for (int i = 0; i < D - 1; ++i) {
        if (ta + i <= tb) issue(ta + i, i);
        cp_async_commit();
    }
    auto step = [&](int t, auto k, auto full) {
        __syncwarp();
        if (t + D - 1 <= tb) issue(t + D - 1, (k + D - 1) % D);
        cp_async_commit();
        cp_async_wait<D - 1>();
        __syncwarp();
        compute(t, k, full);
    };
    int t = ta, slot = 0;
    while (t <= tb) {
        if (slot == 0 && t >= sa && t + D - 1 <= sb) {
            step(t, Slot<0>{}, Full{});
            step(t + 1, Slot<1>{}, Full{});
            step(t + 2, Slot<2>{}, Full{});
            step(t + 3, Slot<3>{}, Full{});
            t += D;
        } else {
            step(t, slot, Edge{});
            ++t;
            slot = slot == D - 1 ? 0 : slot + 1;
        }
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Offset of row t (full: a row inside the slice, no wrap).
template <typename F>
__device__ __forceinline__ long long band_row_at(const BandLane& b, int t, F full) {
    return full ? b.off + (long long)t * b.pitch : band_row(b, t);
}

// k_mgs_fwd on band items (see mg_strip.cuh for the pass).
template <bool UPD>
__global__ void __launch_bounds__(kStripThreads, 4) k_mgb_fwd(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                              const SliceConst* C, SliceState* S, Ptrs<float> P,
                                                              int par, const float* rin, float* rout,
                                                              const float* a2, float* F1, int* pending, int rb,
                                                              int lvl) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    __shared__ BandEdges4 E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 p, 1 r, 2 a^2, 3 z
    BandRing<4>& ring = reinterpret_cast<BandRing<4>*>(strip_dsm)[warp];
    float* z = P.f[RECON_F_Z];
    const float* p = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const BandLane b = band_lane(G, lane, warp, it.slice);
        const SliceGeom* g1p = G1 + it.slice;
        const long long off1 = __ldg(&g1p->off);
        const int pitch1 = __ldg(&g1p->pitch);
        account(P.acct, lvl ? KF_MG_LEVELS : KF_MG_FWD, band_item_px(b, it, rb) * (UPD ? 25 : 9));
        const float bt = mg_bt<float>(*sp, lvl), b4 = 4.f * bt;
        const float al = UPD ? Sc<float>::alpha(*sp) : 0.f;
        const int r0 = min(it.b + b.grp * rb, b.ny), r1 = min(r0 + rb, b.ny);
        float acc = 0.f;
        float4 res_prev = {};
        int buf = 0;
        // odd: wr - r0 is odd (the second row of a restricted pair)
        auto restrict_row = [&](const float4& res, int wr, bool odd) {
            if (odd) {
                if (b.act) {
                    const float c0 = __fadd_rn(__fadd_rn(__fadd_rn(res_prev.x, res_prev.y), res.x), res.y);
                    const float c1 = __fadd_rn(__fadd_rn(__fadd_rn(res_prev.z, res_prev.w), res.z), res.w);
                    *reinterpret_cast<float2*>(F1 + off1 + (long long)(wr >> 1) * pitch1 + (b.x >> 1)) =
                        make_float2(0.25f * c0, 0.25f * c1);
                }
            } else {
                res_prev = res;
            }
        };
        auto sub4 = [](const float4& f, const float4& m) {
            return make_float4(__fsub_rn(f.x, m.x), __fsub_rn(f.y, m.y), __fsub_rn(f.z, m.z), __fsub_rn(f.w, m.w));
        };
        if (!b.idle && r0 < r1) {
            float4 am1 = {}, am2 = {}, rm1 = {}, rm2 = {}, x1m1 = {}, x1m2 = {}, x2m1 = {}, x2m2 = {};
            if constexpr (UPD) {
                // bundle t: p of row t in [r0-3, r1+2]; r, a^2 of row u = t-1 in [r0-2, r1+1]; z of u in [r0, r1)
                auto issue = [&](int t, int k) {
                    if (b.act) cp_async16(&ring.v[k][0][lane], p + band_row(b, t) + b.x);
                    const int u = t - 1;
                    if (u >= r0 - 2 && u <= r1 + 1 && b.act) {
                        const long long ro = band_row(b, u);
                        cp_async16(&ring.v[k][1][lane], rin + ro + b.x);
                        cp_async16(&ring.v[k][2][lane], a2 + ro + b.x);
                        if (u >= r0 && u < r1) cp_async16(&ring.v[k][3][lane], z + ro + b.x);
                    }
                };
                float4 pm2 = {}, pm1 = {};
                float2 lr[3] = {};   // neighbours of pm1, x1m1, x2m1 (exchanged at the end of the step before)
                // steady rows t in [r0+3, r1]: slot k holds bundle t with t - r0 + 3 = k (mod 4), so
                // wr - r0 = t - 3 - r0 has the parity of k
                auto compute = [&](int t, auto k, auto full) {
                    const float4 pt = ring.v[k][0][lane];
                    if (full || t >= r0 - 1) {
                        // row u = t-1: q = M p, r' = r - alpha q, x1 = J r' (and z += alpha p)
                        const int u = t - 1;
                        const float4 au = ring.v[k][2][lane];
                        const float4 q = m_op4(au, pm1, lr[0].x, lr[0].y, pm2, pt, bt);
                        const float4 rn = fma4(-al, q, ring.v[k][1][lane]);
                        const float4 x1 = jac4(rn, au, b4);
                        if ((full || (u >= r0 && u < r1)) && b.act)
                            *reinterpret_cast<float4*>(z + band_row_at(b, u, full) + b.x) =
                                fma4(al, pm1, ring.v[k][3][lane]);
                        if (full || t >= r0 + 1) {
                            // row v = t-2: second pre-smoothing sweep
                            const float4 x2 =
                                sweep4(x1m1, rm1, m_op4(am1, x1m1, lr[1].x, lr[1].y, x1m2, x1, bt), am1, b4);
                            if (full || t >= r0 + 3) {
                                // row w = t-3: residual after pre-smoothing, r' out, r'.r', restriction
                                const int wr = t - 3;
                                const float4 res = sub4(rm2, m_op4(am2, x2m1, lr[2].x, lr[2].y, x2m2, x2, bt));
                                if (b.act) {
                                    *reinterpret_cast<float4*>(rout + band_row_at(b, wr, full) + b.x) = rm2;
                                    acc = dot4(rm2, rm2, acc);
                                }
                                restrict_row(res, wr, full ? (k & 1) != 0 : ((wr - r0) & 1) != 0);
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
                    // p(t), x1(t-1), x2(t-2): their neighbours serve the next step
                    const float4 ex[3] = {pm1, x1m1, x2m1};
                    band_xchg<3>(ex, b, lane, E, buf, lr);
                };
                band_stream(r0 - 3, r1 + 2, r0 + 3, r1, issue, compute);
            } else {
                // bundle t: r, a^2 of row t in [r0-2, r1+1]
                auto issue = [&](int t, int k) {
                    if (b.act) {
                        const long long ro = band_row(b, t);
                        cp_async16(&ring.v[k][1][lane], rin + ro + b.x);
                        cp_async16(&ring.v[k][2][lane], a2 + ro + b.x);
                    }
                };
                float2 lr[2] = {};   // neighbours of x1m1, x2m1 (exchanged at the end of the step before)
                // steady rows t in [r0+2, r1+1]: slot k holds bundle t with t - r0 + 2 = k (mod 4), so
                // w - r0 = t - 2 - r0 has the parity of k
                auto compute = [&](int t, auto k, auto full) {
                    const float4 rt = ring.v[k][1][lane], at = ring.v[k][2][lane];
                    const float4 x1 = jac4(rt, at, b4);
                    if (full || t >= r0) {
                        // row v = t-1: second pre-smoothing sweep
                        const float4 x2 =
                            sweep4(x1m1, rm1, m_op4(am1, x1m1, lr[0].x, lr[0].y, x1m2, x1, bt), am1, b4);
                        if (full || t >= r0 + 2) {
                            // row w = t-2: residual after pre-smoothing, restriction
                            const int wr = t - 2;
                            restrict_row(sub4(rm2, m_op4(am2, x2m1, lr[1].x, lr[1].y, x2m2, x2, bt)), wr,
                                         full ? (k & 1) != 0 : ((wr - r0) & 1) != 0);
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
                    // x1(t), x2(t-1): their neighbours serve the next step
                    const float4 ex[2] = {x1m1, x2m1};
                    band_xchg<2>(ex, b, lane, E, buf, lr);
                };
                band_stream(r0 - 2, r1 + 1, r0 + 2, r1 + 1, issue, compute);
            }
        }
        if (UPD) {
            const float part[1] = {b.act && !b.idle ? acc : 0.f};
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
        } else {
            __syncthreads();   // the next item's edges reuse E
        }
    }
}

// Start of a Z^m solve on the band items of the fine level: k_cg_init and the
// first step's k_mgb_fwd<false> in one pass.  r = rhs - M z (the operator in
// the stencil kernels' rounding sequence, so r equals k_cg_init's bit for
// bit), r out to CG_R, its two pre-smoothing sweeps and the restriction of the
// smoothed residual to level 1 (into F1 on grid G1), and per slice the sums
// r.r, sum a^2 and ||rhs||^2 that initialise the PCG scalars and the
// convergence test as k_cg_init does.  Every active slice takes part: the
// previous solve's cg_done is reset here.
__global__ void __launch_bounds__(kStripThreads, 4) k_mgb_start(ItemList L, const SliceGeom* G,
                                                                const SliceGeom* G1, const SliceConst* C,
                                                                SliceState* S, Ptrs<float> P, float* F1,
                                                                int* pending, int rb) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[3 * 32];
    __shared__ BandEdges4 E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 z, 1 rhs, 2 a^2
    BandRing<3>& ring = reinterpret_cast<BandRing<3>*>(strip_dsm)[warp];
    const float* z = P.f[RECON_F_Z];
    const float* rz = P.f[RECON_F_RHS_Z];
    const float* a2 = P.f[RECON_F_A2];
    float* rout = P.f[RECON_F_CG_R];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active)) continue;
        const BandLane b = band_lane(G, lane, warp, it.slice);
        const SliceGeom* g1p = G1 + it.slice;
        const long long off1 = __ldg(&g1p->off);
        const int pitch1 = __ldg(&g1p->pitch);
        account(P.acct, KF_CG_INIT, band_item_px(b, it, rb) * 17);
        const float bt = Sc<float>::beta_t(*sp), b4 = 4.f * bt;
        const int r0 = min(it.b + b.grp * rb, b.ny), r1 = min(r0 + rb, b.ny);
        float acc_r = 0.f, acc_a = 0.f, acc_b = 0.f;
        float4 res_prev = {};
        int buf = 0;
        auto restrict_row = [&](const float4& res, int wr, bool odd) {
            if (odd) {
                if (b.act) {
                    const float c0 = __fadd_rn(__fadd_rn(__fadd_rn(res_prev.x, res_prev.y), res.x), res.y);
                    const float c1 = __fadd_rn(__fadd_rn(__fadd_rn(res_prev.z, res_prev.w), res.z), res.w);
                    *reinterpret_cast<float2*>(F1 + off1 + (long long)(wr >> 1) * pitch1 + (b.x >> 1)) =
                        make_float2(0.25f * c0, 0.25f * c1);
                }
            } else {
                res_prev = res;
            }
        };
        auto sub4 = [](const float4& f, const float4& m) {
            return make_float4(__fsub_rn(f.x, m.x), __fsub_rn(f.y, m.y), __fsub_rn(f.z, m.z), __fsub_rn(f.w, m.w));
        };
        if (!b.idle && r0 < r1) {
            float4 am1 = {}, am2 = {}, rm1 = {}, rm2 = {}, x1m1 = {}, x1m2 = {}, x2m1 = {}, x2m2 = {};
            float4 zm2 = {}, zm1 = {};
            float2 lr[3] = {};   // neighbours of zm1, x1m1, x2m1 (exchanged at the end of the step before)
            // bundle t: z of row t in [r0-3, r1+2]; rhs, a^2 of row u = t-1 in [r0-2, r1+1]
            auto issue = [&](int t, int k) {
                if (b.act) {
                    cp_async16(&ring.v[k][0][lane], z + band_row(b, t) + b.x);
                    const int u = t - 1;
                    if (u >= r0 - 2 && u <= r1 + 1) {
                        const long long ro = band_row(b, u);
                        cp_async16(&ring.v[k][1][lane], rz + ro + b.x);
                        cp_async16(&ring.v[k][2][lane], a2 + ro + b.x);
                    }
                }
            };
            // steady rows t in [r0+3, r1]: slot k holds bundle t with t - r0 + 3 = k (mod 4)
            auto compute = [&](int t, auto k, auto full) {
                const float4 zt = ring.v[k][0][lane];
                if (full || t >= r0 - 1) {
                    // row u = t-1: r = rhs - M z, x1 = J r
                    const int u = t - 1;
                    const float4 au = ring.v[k][2][lane], bu = ring.v[k][1][lane];
                    const float4 rn = sub4(bu, m_op4(au, zm1, lr[0].x, lr[0].y, zm2, zt, bt));
                    const float4 x1 = jac4(rn, au, b4);
                    if ((full || (u >= r0 && u < r1)) && b.act) {
                        acc_a = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(acc_a, au.x), au.y), au.z), au.w);
                        acc_b = dot4(bu, bu, acc_b);
                    }
                    if (full || t >= r0 + 1) {
                        // row v = t-2: second pre-smoothing sweep
                        const float4 x2 =
                            sweep4(x1m1, rm1, m_op4(am1, x1m1, lr[1].x, lr[1].y, x1m2, x1, bt), am1, b4);
                        if (full || t >= r0 + 3) {
                            // row w = t-3: r out, r.r, residual after pre-smoothing, restriction
                            const int wr = t - 3;
                            const float4 res = sub4(rm2, m_op4(am2, x2m1, lr[2].x, lr[2].y, x2m2, x2, bt));
                            if (b.act) {
                                *reinterpret_cast<float4*>(rout + band_row_at(b, wr, full) + b.x) = rm2;
                                acc_r = dot4(rm2, rm2, acc_r);
                            }
                            restrict_row(res, wr, full ? (k & 1) != 0 : ((wr - r0) & 1) != 0);
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
                zm2 = zm1;
                zm1 = zt;
                // z(t), x1(t-1), x2(t-2): their neighbours serve the next step
                const float4 ex[3] = {zm1, x1m1, x2m1};
                band_xchg<3>(ex, b, lane, E, buf, lr);
            };
            band_stream(r0 - 3, r1 + 2, r0 + 3, r1, issue, compute);
        }
        const bool own = b.act && !b.idle;
        const float part[3] = {own ? acc_r : 0.f, own ? acc_a : 0.f, own ? acc_b : 0.f};
        double a[3];
        block_sum_t<float, 3>(part, a, red);
        double tot[3];
        if (item_reduce<3>(L, w, it.slice, a, tot, red)) {
            SliceState& so = S[it.slice];
            const double tol2 = C[it.slice].cg_tol * C[it.slice].cg_tol;
            set_abar2(so, tot[1] / ((double)b.nx * (double)b.ny));
            so.bb = tot[2];
            so.rr = tot[0];
            so.rr0 = tot[0];
            so.cg_it = 0;
            so.ry = 0.0;
            set_betacg(so, 0.0);
            so.cg_done = (so.bb == 0.0 || !(tot[0] > tol2 * so.bb)) ? 1 : 0;
            if (!so.cg_done) atomicAdd(pending, 1);
        }
    }
}

// k_mgs_up on band items (see mg_strip.cuh for the pass).
template <bool FINE>
__global__ void __launch_bounds__(kStripThreads, 4) k_mgb_up(ItemList L, const SliceGeom* G, const SliceGeom* G1,
                                                             SliceState* S, Ptrs<float> P, const float* r,
                                                             const float* a2, const float* E1, float* out, int rb,
                                                             int lvl) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    __shared__ BandEdges4 E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 r, 1 a^2, 2 e1 (.x, .y: the lane's two coarse cells)
    BandRing<3>& ring = reinterpret_cast<BandRing<3>*>(strip_dsm)[warp];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const BandLane b = band_lane(G, lane, warp, it.slice);
        const SliceGeom* g1p = G1 + it.slice;
        const long long off1 = __ldg(&g1p->off);
        const int pitch1 = __ldg(&g1p->pitch);
        account(P.acct, FINE ? KF_MG_Y : KF_MG_LEVELS, band_item_px(b, it, rb) * 13);
        const float bt = mg_bt<float>(*sp, lvl), b4 = 4.f * bt;
        const int r0 = min(it.b + b.grp * rb, b.ny), r1 = min(r0 + rb, b.ny);
        float acc = 0.f;
        int buf = 0;
        if (!b.idle && r0 < r1) {
            // bundle t: r, a^2 of row t in [r0-3, r1+2]; e1 under row u = t-1 in [r0-2, r1+1]
            auto issue = [&](int t, int k) {
                if (b.act) {
                    const long long ro = band_row(b, t);
                    cp_async16(&ring.v[k][0][lane], r + ro + b.x);
                    cp_async16(&ring.v[k][1][lane], a2 + ro + b.x);
                    const int u = t - 1;
                    if (u >= r0 - 2 && u <= r1 + 1) {
                        const long long co = off1 + (long long)(wrap_near(u, b.ny) >> 1) * pitch1;
                        cp_async_elem<8>(&ring.v[k][2][lane], E1 + co + (b.x >> 1));
                    }
                }
            };
            float4 rm1 = {}, rm2 = {}, rm3 = {}, am1 = {}, am2 = {}, am3 = {};
            float4 x1m1 = {}, x1m2 = {}, xm1 = {}, xm2 = {}, xpm1 = {}, xpm2 = {};
            float2 lr[3] = {};   // neighbours of x1m1, xm1, xpm1 (exchanged at the end of the step before)
            // steady rows t in [r0+3, r1+2]
            auto compute = [&](int t, auto k, auto full) {
                const float4 rt = ring.v[k][0][lane], at = ring.v[k][1][lane];
                const float4 x1 = jac4(rt, at, b4);
                if (full || t >= r0 - 1) {
                    // row u = t-1: second pre-smoothing sweep, then the prolonged correction
                    float4 x = sweep4(x1m1, rm1, m_op4(am1, x1m1, lr[0].x, lr[0].y, x1m2, x1, bt), am1, b4);
                    const float4 e = ring.v[k][2][lane];
                    x.x = __fadd_rn(x.x, e.x);
                    x.y = __fadd_rn(x.y, e.x);
                    x.z = __fadd_rn(x.z, e.y);
                    x.w = __fadd_rn(x.w, e.y);
                    if (full || t >= r0 + 1) {
                        // row v = t-2: first post-smoothing sweep
                        const float4 xp = sweep4(xm1, rm2, m_op4(am2, xm1, lr[1].x, lr[1].y, xm2, x, bt), am2, b4);
                        if (full || t >= r0 + 3) {
                            // row w = t-3: second post-smoothing sweep, out (and r.y)
                            const float4 y =
                                sweep4(xpm1, rm3, m_op4(am3, xpm1, lr[2].x, lr[2].y, xpm2, xp, bt), am3, b4);
                            if (b.act) {
                                *reinterpret_cast<float4*>(out + band_row_at(b, t - 3, full) + b.x) = y;
                                if (FINE) acc = dot4(rm3, y, acc);
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
                // x1(t), x(t-1), xp(t-2): their neighbours serve the next step
                const float4 ex[3] = {x1m1, xm1, xpm1};
                band_xchg<3>(ex, b, lane, E, buf, lr);
            };
            band_stream(r0 - 3, r1 + 2, r0 + 3, r1 + 2, issue, compute);
        }
        if (FINE) {
            const float part[1] = {b.act && !b.idle ? acc : 0.f};
            double a[1];
            block_sum_t<float, 1>(part, a, red);
            double tot[1];
            if (item_reduce<1>(L, w, it.slice, a, tot, red)) {
                SliceState& so = S[it.slice];
                set_betacg(so, (so.cg_it == 0) ? 0.0 : tot[0] / so.ry);
                so.ry = tot[0];
            }
        } else {
            __syncthreads();   // the next item's edges reuse E
        }
    }
}

// k_mgs_pq on band items (see mg_strip.cuh for the pass).
template <bool STOREQ>
__global__ void __launch_bounds__(kStripThreads, 4) k_mgb_pq(ItemList L, const SliceGeom* G, SliceState* S,
                                                             Ptrs<float> P, int par, int rb) {
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ double red[32];
    __shared__ BandEdges4 E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fields: 0 y, 1 p_old, 2 a^2
    BandRing<3>& ring = reinterpret_cast<BandRing<3>*>(strip_dsm)[warp];
    const float* yf = P.f[RECON_F_CG_Y];
    const float* pold = P.f[par ? RECON_F_CG_P1 : RECON_F_CG_P0];
    float* pnew = P.f[par ? RECON_F_CG_P0 : RECON_F_CG_P1];
    const float* a2 = P.f[RECON_F_A2];
    float* qo = P.f[RECON_F_CG_Q];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active) || __ldg(&sp->cg_done)) continue;
        const BandLane b = band_lane(G, lane, warp, it.slice);
        const bool first = __ldg(&sp->cg_it) == 0;
        account(P.acct, KF_MG_PQ, band_item_px(b, it, rb) * (first ? 12 : 16));
        const float bc = first ? 0.f : Sc<float>::betacg(*sp), bt = Sc<float>::beta_t(*sp);
        const int r0 = min(it.b + b.grp * rb, b.ny), r1 = min(r0 + rb, b.ny);
        float acc = 0.f;
        int buf = 0;
        if (!b.idle && r0 < r1) {
            // bundle t: y, p_old of row t in [r0-1, r1]; a^2 of row t-1 in [r0, r1-1]
            auto issue = [&](int t, int k) {
                if (b.act) {
                    const long long ro = band_row(b, t);
                    cp_async16(&ring.v[k][0][lane], yf + ro + b.x);
                    if (!first) cp_async16(&ring.v[k][1][lane], pold + ro + b.x);
                    if (t - 1 >= r0 && t - 1 < r1) cp_async16(&ring.v[k][2][lane], a2 + band_row(b, t - 1) + b.x);
                }
            };
            float4 pm2 = {}, pm1 = {};
            float2 lr[1] = {};   // neighbours of pm1 (exchanged at the end of the step before)
            // steady rows t in [r0+1, r1-1]
            auto compute = [&](int t, auto k, auto full) {
                float4 pt = ring.v[k][0][lane];
                if (!first) pt = fma4(bc, ring.v[k][1][lane], pt);
                if ((full || (t >= r0 && t < r1)) && b.act)
                    *reinterpret_cast<float4*>(pnew + band_row_at(b, t, full) + b.x) = pt;
                if (full || t >= r0 + 1) {
                    // row t-1: q = M p, p.q
                    const float4 q = m_op4(ring.v[k][2][lane], pm1, lr[0].x, lr[0].y, pm2, pt, bt);
                    if (b.act) {
                        acc = dot4(pm1, q, acc);
                        if (STOREQ) *reinterpret_cast<float4*>(qo + band_row_at(b, t - 1, full) + b.x) = q;
                    }
                }
                pm2 = pm1;
                pm1 = pt;
                // p(t): its neighbours serve the next step
                const float4 ex[1] = {pm1};
                band_xchg<1>(ex, b, lane, E, buf, lr);
            };
            band_stream(r0 - 1, r1, r0 + 1, r1 - 1, issue, compute);
        }
        const float part[1] = {b.act && !b.idle ? acc : 0.f};
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
