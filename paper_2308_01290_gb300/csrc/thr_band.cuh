// The threshold and right-hand-side pass of Algorithm 1 (k_thr_rhs without
// the statistics) for FP32 slices up to kBandMaxW columns wide, as a
// register-streaming band kernel on the layout of mg_band.cuh: eq. sol_hv for
// the four maps (periodic forward differences, reading R6; tie -> 0, R7), the
// divergences of the kept gradients, and the right-hand sides of the f1 / f2
// closed forms (image domain) or of the sinogram-domain normal equations.
// Included by solver.cu after mg_band.cuh.
//
// Each pixel's gradient (dx, dy) = (m[y][x+1] - m[y][x], m[y+1][x] - m[y][x])
// and its keep decision are formed once: the divergence at (y, x) takes the
// kept h of (y, x - 1) from the lane to the left and the kept v of (y - 1, x)
// from the row walked before, (h(y, x-1) - h(y, x)) + (v(y-1, x) - v(y, x)),
// with the same operations and roundings as k_thr_rhs.  A warp walks rows
// r0 - 1 .. r1 of its band (one halo row above for v, one below for dy); the
// right neighbours of the four maps and the left neighbours of the four h
// rows cross the warp edges through shared memory, one barrier for all four
// maps each.
#pragma once

namespace recon {

constexpr int kThrRows = 32;   // rows a warp walks per band item of the threshold pass

// Left (l) and right (r) neighbours of the lane's four columns of each of
// c[0..3], one barrier.  LEFT / RIGHT: which sides are needed.
template <bool LEFT, bool RIGHT>
__device__ __forceinline__ void band_lr4(const float4 (&c)[4], const BandLane& b, int lane, BandEdges4& E, int& buf,
                                         float (&l)[4], float (&r)[4]) {
    float4(&e)[kStripWarps][2] = E.e[buf][b.grp];
    if (RIGHT && lane == 0) e[b.wg][0] = make_float4(c[0].x, c[1].x, c[2].x, c[3].x);
    if (LEFT && lane == b.lastw) e[b.wg][1] = make_float4(c[0].w, c[1].w, c[2].w, c[3].w);
    band_bar(b.grp, 32 * b.G);
    if (LEFT) {
        const float4 o = e[b.lsrc][1];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float up = __shfl_up_sync(0xffffffffu, c[k].w, 1);
            l[k] = lane == 0 ? f4_get(o, k) : up;
        }
    }
    if (RIGHT) {
        const float4 o = e[b.rsrc][0];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dn = __shfl_down_sync(0xffffffffu, c[k].x, 1);
            r[k] = lane == b.lastw ? f4_get(o, k) : dn;
        }
    }
    buf ^= 1;
}

// Kept gradient of a pixel (eq. sol_hv): (dx, dy) when dx^2 + dy^2 > thr, else 0.
__device__ __forceinline__ void kept(float c, float right, float below, float thr, float& h, float& v) {
    const float dx = __fsub_rn(right, c), dy = __fsub_rn(below, c);
    const bool k = keep_grad(dx, dy, thr);
    h = k ? dx : 0.f;
    v = k ? dy : 0.f;
}

template <bool SINO>
__global__ void __launch_bounds__(kStripThreads, SINO ? 3 : 4) k_thr_band(ItemList L, const SliceGeom* G,
                                                                          const SliceConst* C, const SliceState* S,
                                                                          Ptrs<float> P, int rb) {
    constexpr int NF = SINO ? 8 : 6;   // f1, f2, rho_e, z; uL, uH (; A^T A f1, A^T A f2)
    extern __shared__ __align__(16) unsigned char strip_dsm[];
    __shared__ BandEdges4 E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BandRing<NF>& ring = reinterpret_cast<BandRing<NF>*>(strip_dsm)[warp];
    const float* mp[4] = {P.f[RECON_F_F1], P.f[RECON_F_F2], P.f[RECON_F_RHO], P.f[RECON_F_Z]};
    const float* uLp = P.f[RECON_F_MUL];
    const float* uHp = P.f[RECON_F_MUH];
    const float* g1p = P.f[RECON_F_A2];
    const float* g2p = P.f[RECON_F_RHS_Z];
    for (int w = blockIdx.x; w < L.n_items; w += gridDim.x) {
        const Item it = L.items[w];
        const SliceState* sp = S + it.slice;
        if (!__ldg(&sp->active)) continue;
        const BandLane b = band_lane(G, lane, warp, it.slice);
        account(P.acct, KF_THR_RHS, band_item_px(b, it, rb) * (SINO ? 48 : 40));
        const SliceConst& c = C[it.slice];
        const float thr = sp->thr_f, beta = Sc<float>::beta(*sp), beta_t = Sc<float>::beta_t(*sp);
        const float A00 = c.fk[KC_A00], A01 = c.fk[KC_A01], A10 = c.fk[KC_A10], A11 = c.fk[KC_A11];
        const float b00 = c.fk[KC_B00], b01 = c.fk[KC_B01], b10 = c.fk[KC_B10], b11 = c.fk[KC_B11];
        const float P1 = c.fk[KC_P1], P2 = c.fk[KC_P2], PSI1 = c.fk[KC_PSI1], PSI2 = c.fk[KC_PSI2];
        const float c12 = c.fk[KC_C12], ag = c.fk[KC_SINO_AG], bc = c.fk[KC_SINO_BC];
        const int order = c.order;
        const int r0 = min(it.b + b.grp * rb, b.ny), r1 = min(r0 + rb, b.ny);
        int buf = 0;
        if (!b.idle && r0 < r1) {
            // bundle t: the four maps of row t in [r0-1, r1]; uL, uH (, G1, G2) of row t-1 in [r0, r1)
            auto issue = [&](int t, int k) {
                if (b.act) {
                    const long long ro = band_row(b, t);
#pragma unroll
                    for (int m = 0; m < 4; ++m) cp_async16(&ring.v[k][m][lane], mp[m] + ro + b.x);
                    if (t - 1 >= r0 && t - 1 < r1) {
                        const long long ru = band_row(b, t - 1);
                        cp_async16(&ring.v[k][4][lane], uLp + ru + b.x);
                        cp_async16(&ring.v[k][5][lane], uHp + ru + b.x);
                        if (SINO) {
                            cp_async16(&ring.v[k][NF - 2][lane], g1p + ru + b.x);
                            cp_async16(&ring.v[k][NF - 1][lane], g2p + ru + b.x);
                        }
                    }
                }
            };
            float4 mu[4] = {}, vprev[4] = {};   // maps of row t-1; kept v of row t-2
            auto compute = [&](int t, auto k, auto full) {
                float4 mt[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) mt[m] = ring.v[k][m][lane];
                if (full || t >= r0) {
                    // row u = t-1: kept gradients of the four maps
                    const int u = t - 1;
                    float rn[4], ln[4], hl[4];
                    band_lr4<false, true>(mu, b, lane, E, buf, ln, rn);
                    float4 h[4], v[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        kept(mu[m].x, mu[m].y, mt[m].x, thr, h[m].x, v[m].x);
                        kept(mu[m].y, mu[m].z, mt[m].y, thr, h[m].y, v[m].y);
                        kept(mu[m].z, mu[m].w, mt[m].z, thr, h[m].z, v[m].z);
                        kept(mu[m].w, rn[m], mt[m].w, thr, h[m].w, v[m].w);
                    }
                    band_lr4<true, false>(h, b, lane, E, buf, hl, rn);
                    if (full || u >= r0) {
                        // divergence (h(x-1) - h) + (v(y-1) - v) of each map at row u
                        float4 dv[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            dv[m].x = __fadd_rn(__fsub_rn(hl[m], h[m].x), __fsub_rn(vprev[m].x, v[m].x));
                            dv[m].y = __fadd_rn(__fsub_rn(h[m].x, h[m].y), __fsub_rn(vprev[m].y, v[m].y));
                            dv[m].z = __fadd_rn(__fsub_rn(h[m].y, h[m].z), __fsub_rn(vprev[m].z, v[m].z));
                            dv[m].w = __fadd_rn(__fsub_rn(h[m].z, h[m].w), __fsub_rn(vprev[m].w, v[m].w));
                        }
                        const float4 uL = ring.v[k][4][lane], uH = ring.v[k][5][lane];
                        float4 G1 = {}, G2 = {};
                        if (SINO) {
                            G1 = ring.v[k][NF - 2][lane];
                            G2 = ring.v[k][NF - 1][lane];
                        }
                        float4 o0, o1, o2, o3;
                        auto px = [&](float f1, float f2, float rho, float z, float uL_, float uH_, float G1_,
                                      float G2_, float d0, float d1, float d2, float d3, float& x0, float& x1,
                                      float& x2, float& x3) {
                            const float M1 = rho * (P1 * z + PSI1);
                            const float M2 = rho * (P2 * z + PSI2);
                            if (!SINO) {
                                const float base1 = A00 * uL_ + A01 * uH_ + b00 * M1 + b01 * M2;
                                const float base2 = A10 * uL_ + A11 * uH_ + b10 * M1 + b11 * M2;
                                x0 = base1 - c12 * f2 + beta * d0;
                                x1 = (order ? base2 : base2 - c12 * f1) + beta * d1;
                            } else {
                                x0 = uL_ + b00 * M1 + b01 * M2 - ag * G2_ - bc * f2 + beta * d0;
                                x1 = uH_ + b10 * M1 + b11 * M2 - ag * G1_ - bc * f1 + beta * d1;
                            }
                            x2 = beta_t * d2;
                            x3 = beta_t * d3;
                        };
                        px(mu[0].x, mu[1].x, mu[2].x, mu[3].x, uL.x, uH.x, G1.x, G2.x, dv[0].x, dv[1].x, dv[2].x,
                           dv[3].x, o0.x, o1.x, o2.x, o3.x);
                        px(mu[0].y, mu[1].y, mu[2].y, mu[3].y, uL.y, uH.y, G1.y, G2.y, dv[0].y, dv[1].y, dv[2].y,
                           dv[3].y, o0.y, o1.y, o2.y, o3.y);
                        px(mu[0].z, mu[1].z, mu[2].z, mu[3].z, uL.z, uH.z, G1.z, G2.z, dv[0].z, dv[1].z, dv[2].z,
                           dv[3].z, o0.z, o1.z, o2.z, o3.z);
                        px(mu[0].w, mu[1].w, mu[2].w, mu[3].w, uL.w, uH.w, G1.w, G2.w, dv[0].w, dv[1].w, dv[2].w,
                           dv[3].w, o0.w, o1.w, o2.w, o3.w);
                        if (b.act) {
                            const long long ro = band_row_at(b, u, full) + b.x;
                            *reinterpret_cast<float4*>(P.f[RECON_F_RHS_F1] + ro) = o0;
                            *reinterpret_cast<float4*>(P.f[RECON_F_RHS_F2] + ro) = o1;
                            *reinterpret_cast<float4*>(P.f[RECON_F_DIV_RHO] + ro) = o2;
                            *reinterpret_cast<float4*>(P.f[RECON_F_DIV_Z] + ro) = o3;
                        }
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) vprev[m] = v[m];
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) mu[m] = mt[m];
            };
            band_stream(r0 - 1, r1, r0 + 1, r1, issue, compute);
        }
        __syncthreads();   // the next item's edges reuse E
    }
}

}  // namespace recon
