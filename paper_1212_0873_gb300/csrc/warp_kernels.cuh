// Warp-cooperative persistent form of PCDM1 for long columns (Algorithm 1,
// step 4, the step of eq. (h(x)) with w = L).  Included at the end of
// pcdm_kernels.cuh.
//
// Position j of S_k belongs to warp j mod (warps of the grid), which owns the
// positions gw, gw + nw, gw + 2 nw, ... (at most 32: lane t owns the t-th), so
// tau must not exceed 32 times the warps of the grid.  The 32 lanes share each
// of the warp's columns, one column at a time:
//   load     lane l reads entries 2l, 2l+1 of each run of 64 entries of the
//            next column (row indices and values with 8- and 16-byte loads:
//            every request of the warp covers consecutive bytes) while the
//            current column is processed; a bulk L2 prefetch issued kWarpAhead
//            columns earlier has asked for the column;
//   gather   g at the next column's rows, issued before the products of the
//            current column (whose gathers went out one step earlier);
//   reduce   the partial sums of eight columns are summed over the warp by a
//            transposed butterfly (9 exchange-and-add steps for 8 columns
//            instead of 40), which leaves each column's gradient with its
//            owner lane;
//   step     the owner lanes take their steps side by side (FP64), store x_i;
//   scatter  the warp adds A_i h_i of the moving coordinates (about 1% of
//            LASSO's) into the other residual buffer, rereading the column.
// The residual is double-buffered as in the pipelined kernel: iteration k
// gathers from buffer k & 1 and adds the steps of iterations k-1 and k into the
// other one, so a single bounded grid barrier separates the iterations.
#pragma once

#include <type_traits>

namespace pcdm {

// Two consecutive stored values (the first at an even entry) as the accumulation dtype.
__device__ __forceinline__ void ld_pair(const double *p, double &v0, double &v1)
{
    const double2 d = __ldcs(reinterpret_cast<const double2 *>(p));
    v0 = d.x;
    v1 = d.y;
}
__device__ __forceinline__ void ld_pair(const float *p, float &v0, float &v1)
{
    const float2 d = __ldcs(reinterpret_cast<const float2 *>(p));
    v0 = d.x;
    v1 = d.y;
}
__device__ __forceinline__ void ld_pair(const bf16_t *p, float &v0, float &v1)
{
    const uint32_t u = __ldcs(reinterpret_cast<const unsigned int *>(p));
    v0 = __uint_as_float(u << 16);
    v1 = __uint_as_float(u & 0xFFFF0000u);
}

// Sum over the warp of eight per-lane partials p[0..7]; lanes 4c .. 4c+3 return
// the total of partial c.  The first three levels halve what a lane keeps (lanes
// with bit 4 set keep partials 4..7 and send 0..3 to their partner, and so on
// with bits 3 and 2), the last two finish the sums over the remaining lanes.
// The four lanes of a partial end with the same value (each top-level add has
// the same two operands).
template <typename T>
__device__ __forceinline__ T transposed_sum8(const T (&p)[8], int lane)
{
    const unsigned full = 0xFFFFFFFFu;
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
    T q[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = (b4 ? p[4 + c] : p[c]) + __shfl_xor_sync(full, b4 ? p[c] : p[4 + c], 16);
    T r[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) r[c] = (b3 ? q[2 + c] : q[c]) + __shfl_xor_sync(full, b3 ? q[c] : q[2 + c], 8);
    T s = (b2 ? r[1] : r[0]) + __shfl_xor_sync(full, b2 ? r[0] : r[1], 4);
    s += __shfl_xor_sync(full, s, 2);
    s += __shfl_xor_sync(full, s, 1);
    return s;
}

// The same for two partials: lanes 16c .. 16c+15 return the total of partial c.
template <typename T>
__device__ __forceinline__ T transposed_sum2(const T (&p)[2], int lane)
{
    const unsigned full = 0xFFFFFFFFu;
    const bool b4 = (lane & 16) != 0;
    T s = (b4 ? p[1] : p[0]) + __shfl_xor_sync(full, b4 ? p[0] : p[1], 16);
    s += __shfl_xor_sync(full, s, 8);
    s += __shfl_xor_sync(full, s, 4);
    s += __shfl_xor_sync(full, s, 2);
    s += __shfl_xor_sync(full, s, 1);
    return s;
}

// Transposed reduction of four per-lane values with max (the certificate's
// largest operand image): lanes 8c .. 8c+7 return the maximum of value c.
__device__ __forceinline__ float transposed_max4(const float (&p)[4], int lane)
{
    const unsigned full = 0xFFFFFFFFu;
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
    float q[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) q[c] = fmaxf(b4 ? p[2 + c] : p[c], __shfl_xor_sync(full, b4 ? p[c] : p[2 + c], 16));
    float s = fmaxf(b3 ? q[1] : q[0], __shfl_xor_sync(full, b3 ? q[0] : q[1], 8));
    s = fmaxf(s, __shfl_xor_sync(full, s, 4));
    s = fmaxf(s, __shfl_xor_sync(full, s, 2));
    s = fmaxf(s, __shfl_xor_sync(full, s, 1));
    return s;
}

// The same for four partials: lanes 8c .. 8c+7 return the total of partial c
// (6 exchange-and-add steps for 4 columns; fewer registers than eight).
template <typename T>
__device__ __forceinline__ T transposed_sum4(const T (&p)[4], int lane)
{
    const unsigned full = 0xFFFFFFFFu;
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
    T q[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) q[c] = (b4 ? p[2 + c] : p[c]) + __shfl_xor_sync(full, b4 ? p[c] : p[2 + c], 16);
    T s = (b3 ? q[1] : q[0]) + __shfl_xor_sync(full, b3 ? q[0] : q[1], 8);
    s += __shfl_xor_sync(full, s, 4);
    s += __shfl_xor_sync(full, s, 2);
    s += __shfl_xor_sync(full, s, 1);
    return s;
}

// A group's new last entry (the others move down one place).
template <typename T, int N>
__device__ __forceinline__ void shift_in(T (&v)[N], T x)
{
#pragma unroll
    for (int c = 0; c < N - 1; ++c) v[c] = v[c + 1];
    v[N - 1] = x;
}

// Total of entry c of a group of N (8 or 4) per-lane values over the warp, in
// the lanes that own column c of the group (lane mod N == c).
template <typename T, int N>
__device__ __forceinline__ T group_total(const T (&v)[N], int lane)
{
    if constexpr (N == 8)
        return __shfl_sync(0xFFFFFFFFu, transposed_sum8(v, lane), 4 * (lane & 7));
    else
        return __shfl_sync(0xFFFFFFFFu, transposed_sum4(v, lane), 8 * (lane & 3));
}

// ZC (FP64 form of LASSO): the gradients are first summed in FP32 over images of
// the operands' high words (ZeroCert); a column whose bound shows |a_i^T g| <=
// lambda at x_i = 0 takes the zero step with no FP64 instruction, the others
// (x_i != 0, |grad| near lambda) are summed again in FP64 from memory.  Each
// product of the FP32 sums passes through its lane's FMAs and the five levels
// of the warp reduction, at most c + 5 roundings for a column of c entries, so
// the bound is taken with c + 5 in place of c.
template <typename VT, typename XT, int GM = 0, bool ZC = false>
__global__ void __launch_bounds__(kWarpMaxBlock, 1) k_fused_warp(const IterArgs<VT, XT> a, int64_t k0, int64_t iters)
{
    constexpr bool CERT = sizeof(XT) == 8 && GM == 0 && ZC;
    using EV = std::conditional_t<CERT, uint32_t, XT>;   // a value or gathered g as held: its high word, or itself
    constexpr int R = CERT ? 3 : warp_rounds<XT>();     // runs of 64 entries held in registers per column
    constexpr int RUN = 64;
    constexpr unsigned FULL = 0xFFFFFFFFu;
    constexpr int G = pad_granule<VT>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int64_t nw = int64_t(gridDim.x) * wpb;
    const int64_t gw = int64_t(blockIdx.x) * wpb + warp;
    const int T = a.tau > gw ? int(min(int64_t(32), (a.tau - gw + nw - 1) / nw)) : 0;   // positions of this warp
    const int64_t j = gw + int64_t(lane) * nw;                                            // lane t: position t
    const bool mine = lane < T;
    Counters cnt;
    const uint64_t pf = l2_evict_first();   // descriptors, x
    const uint64_t pl = l2_evict_last();    // the residual buffers
    const float lamf = __double2float_rd(a.lambda);
    auto gbuf = [&](int64_t kk) { return (kk & 1) ? a.g2 : a.g; };

    // Lane t: the column of its position in the current (c_) and the next (n_)
    // iteration, and the previous iteration's column and step (still owed to
    // the buffer the current iteration gathers from).
    int32_t c_i = 0, n_i = 0;
    Col<XT> c_d, n_d, p_d;
    c_d.pbeg = n_d.pbeg = p_d.pbeg = 0;
    c_d.cnt = n_d.cnt = p_d.cnt = 0;
    c_d.invL = n_d.invL = p_d.invL = XT(0);
    XT h_prev = XT(0);
    if (mine) {
        c_i = ldcg(sample_buf(a, k0) + j);
        c_d = load_col(a.desc, c_i, pf);
    }
    // Bring a column's entries (padded run) into L2 ahead of its loads.
    auto prefetch_col = [&](const Col<XT> &d) {
        if (d.cnt > 0) {
            const uint32_t pc = uint32_t((d.cnt + G - 1) / G * G);
            prefetch_l2_bulk(a.prow + d.pbeg, pc * 4u);
            prefetch_l2_bulk(a.pval + d.pbeg, pc * uint32_t(sizeof(VT)));
        }
    };
    if (lane < kWarpAhead && mine) prefetch_col(c_d);

    // Runs 0 .. R-1 of a column: lane l holds entries 64r + 2l, 64r + 2l + 1
    // (the guards on 64r are warp-uniform; entries past the column's end are
    // read from its padding or the next column and never used).
    auto load_runs = [&](int64_t pbeg, int ccnt, int32_t (&row)[R][2], EV (&val)[R][2]) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (RUN * r < ccnt) {
                const int e = RUN * r + 2 * lane;
                const int2 rr = __ldcs(reinterpret_cast<const int2 *>(a.prow + pbeg + e));
                row[r][0] = rr.x;
                row[r][1] = rr.y;
                if constexpr (CERT) {
                    const uint4 u = __ldcs(reinterpret_cast<const uint4 *>(a.pval + pbeg + e));
                    val[r][0] = u.y;
                    val[r][1] = u.w;
                } else {
                    ld_pair(a.pval + pbeg + e, val[r][0], val[r][1]);
                }
            }
        }
    };
    auto gather_one = [&](const XT *gk, int32_t row) -> EV {
        if constexpr (CERT)
            return ldcg_hi_hint(gk + row, pl);
        else
            return ldcg_hint(gk + row, pl);
    };
    auto gather_runs = [&](const XT *gk, int ccnt, const int32_t (&row)[R][2], EV (&gv)[R][2]) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (RUN * r < ccnt) {
                const int e = RUN * r + 2 * lane;
                gv[r][0] = e < ccnt ? gather_one(gk, row[r][0]) : EV(0);
                gv[r][1] = e + 1 < ccnt ? gather_one(gk, row[r][1]) : EV(0);
            }
        }
    };
    // This lane's share of a column: the FP32 certificate sums (CERT) or a_i^T phi(g).
    using Part = std::conditional_t<CERT, ZeroCert, XT>;
    auto add_entry = [&](Part &p, EV v, EV g) {
        if constexpr (CERT)
            p.add(v, g);
        else
            p = fma(v, grad_map<GM>(g), p);
    };
    auto dot_runs = [&](int ccnt, const EV (&val)[R][2], const EV (&gv)[R][2]) {
        Part p = Part();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (RUN * r < ccnt) {
                const int e = RUN * r + 2 * lane;
                if (e < ccnt) add_entry(p, val[r][0], gv[r][0]);
                if (e + 1 < ccnt) add_entry(p, val[r][1], gv[r][1]);
            }
        }
        return p;
    };
    // Entries past the first R runs (columns longer than 64 R entries), run by run.
    auto dot_tail = [&](const XT *gk, int64_t pbeg, int ccnt, Part &p) {
        for (int cs = RUN * R; cs < ccnt; cs += RUN) {
            const int e = cs + 2 * lane;
            if (e < ccnt) {
                int32_t row[1][2];
                EV val[1][2];
                const int2 rr = __ldcs(reinterpret_cast<const int2 *>(a.prow + pbeg + e));
                row[0][0] = rr.x;
                row[0][1] = rr.y;
                if constexpr (CERT) {
                    const uint4 u = __ldcs(reinterpret_cast<const uint4 *>(a.pval + pbeg + e));
                    val[0][0] = u.y;
                    val[0][1] = u.w;
                } else {
                    ld_pair(a.pval + pbeg + e, val[0][0], val[0][1]);
                }
                const EV g0 = gather_one(gk, row[0][0]);
                const EV g1 = e + 1 < ccnt ? gather_one(gk, row[0][1]) : EV(0);
                add_entry(p, val[0][0], g0);
                if (e + 1 < ccnt) add_entry(p, val[0][1], g1);
            }
        }
    };
    // Column partials enter groups of GS (eight, four in FP64 to save registers);
    // a full group (or the last column) is summed over the warp and each
    // column's result goes to its owner lane: the gradient, or (CERT) the three
    // certificate sums.
    constexpr int GS = sizeof(XT) == 8 ? 4 : 8;
    XT acc[GS], grad = XT(0);
    float zs[GS], za[GS], zm[GS], own_s = 0.f, own_a = 0.f, own_m = 0.f;
    int closed = 0;
    auto push = [&](const Part &p) {
        if constexpr (CERT) {
            shift_in(zs, p.acc);
            shift_in(za, p.sabs);
            shift_in(zm, p.mx);
        } else {
            shift_in(acc, p);
        }
    };
    auto close_col = [&](const Part &part) {
        push(part);
        if ((closed & (GS - 1)) == GS - 1 || closed == T - 1) {
            for (int z = closed & (GS - 1); z < GS - 1; ++z) push(Part());   // the last group: zeros after it
            const bool owner = lane / GS == closed / GS;
            if constexpr (CERT) {
                const float s = group_total(zs, lane), ab = group_total(za, lane);
                const float mx = __shfl_sync(FULL, transposed_max4(zm, lane), 8 * (lane & 3));
                if (owner) {
                    own_s = s;
                    own_a = ab;
                    own_m = mx;
                }
            } else {
                const XT v = group_total(acc, lane);
                if (owner) grad = v;
            }
        }
        ++closed;
    };
    // The rereading passes take QS columns of a lane mask at a time (the q-th
    // lowest set lane in slot q; an empty slot has no entries), QB runs of 32
    // entries of each per batch, so that their loads and gathers are in flight
    // together: two columns with an FP32 residual, one (two runs per batch) in
    // FP64, whose registers would otherwise spill.
    constexpr int QS = sizeof(XT) == 8 ? 1 : 2;
    constexpr int QB = sizeof(XT) == 8 ? 2 : 1;
    auto take = [&](unsigned &m, const Col<XT> &d, int (&tq)[QS], int64_t (&pbq)[QS], int (&ccq)[QS]) {
#pragma unroll
        for (int q = 0; q < QS; ++q) {
            const bool any = m != 0u;
            const int t = any ? __ffs(int(m)) - 1 : 0;
            if (any) m &= m - 1u;
            tq[q] = any ? t : -1;
            pbq[q] = __shfl_sync(FULL, d.pbeg, t);
            const int cc = __shfl_sync(FULL, d.cnt, t);
            ccq[q] = any ? cc : 0;
        }
    };
    // FP64 gradient of each column in mask m (the columns the certificate did
    // not decide), read again from memory; the sum goes to the owner lane.
    auto fp64_grads = [&](unsigned m, const XT *gk) {
        while (m) {
            int tq[QS], ccq[QS];
            int64_t pbq[QS];
            take(m, c_d, tq, pbq, ccq);
            int ccmax = 0;
#pragma unroll
            for (int q = 0; q < QS; ++q) ccmax = max(ccmax, ccq[q]);
            XT p[QS];
#pragma unroll
            for (int q = 0; q < QS; ++q) p[q] = XT(0);
            for (int cs = 0; cs < ccmax; cs += 32 * QB) {
                // a batch: every load, then every gather, then the products
                int32_t rr[QS][QB];
                XT vv[QS][QB], gg[QS][QB];
#pragma unroll
                for (int q = 0; q < QS; ++q)
#pragma unroll
                    for (int b = 0; b < QB; ++b) {
                        const int e = cs + lane + 32 * b;
                        rr[q][b] = e < ccq[q] ? __ldg(a.prow + pbq[q] + e) : 0;
                        vv[q][b] = e < ccq[q] ? XT(ldv(a.pval + pbq[q] + e)) : XT(0);
                    }
#pragma unroll
                for (int q = 0; q < QS; ++q)
#pragma unroll
                    for (int b = 0; b < QB; ++b)
                        gg[q][b] = cs + lane + 32 * b < ccq[q] ? ldcg_hint(gk + rr[q][b], pl) : XT(0);
#pragma unroll
                for (int q = 0; q < QS; ++q)
#pragma unroll
                    for (int b = 0; b < QB; ++b) p[q] = fma(vv[q][b], gg[q][b], p[q]);
            }
            if constexpr (QS == 1) {
                const XT v = warp_sum(p[0]);
                if (lane == tq[0]) grad = v;
            } else {
                // the two sums over the warp at once: slot q's total in lanes 16q .. 16q+15
                const XT tot = transposed_sum2(p, lane);
#pragma unroll
                for (int q = 0; q < QS; ++q) {
                    const XT v = __shfl_sync(FULL, tot, 16 * q);
                    if (lane == tq[q]) grad = v;
                }
            }
        }
    };
    // The warp adds A_i h_i of its moving coordinates (d, hv of lane t) into gdst.
    auto scatter_owned = [&](const Col<XT> &d, XT hv, XT *gdst) {
        unsigned m = __ballot_sync(FULL, mine && !is_zero_bits(hv));
        while (m) {
            int tq[QS], ccq[QS];
            int64_t pbq[QS];
            take(m, d, tq, pbq, ccq);
            XT hq[QS];
            int ccmax = 0;
#pragma unroll
            for (int q = 0; q < QS; ++q) {
                hq[q] = __shfl_sync(FULL, hv, tq[q] < 0 ? 0 : tq[q]);
                ccmax = max(ccmax, ccq[q]);
            }
            for (int cs = 0; cs < ccmax; cs += 32 * QB) {
                // a batch: every load, then the atomic adds
                int32_t rr[QS][QB];
                XT vv[QS][QB];
#pragma unroll
                for (int q = 0; q < QS; ++q)
#pragma unroll
                    for (int b = 0; b < QB; ++b) {
                        const int e = cs + lane + 32 * b;
                        rr[q][b] = e < ccq[q] ? __ldg(a.prow + pbq[q] + e) : 0;
                        vv[q][b] = e < ccq[q] ? XT(ldv(a.pval + pbq[q] + e)) : XT(0);
                    }
#pragma unroll
                for (int q = 0; q < QS; ++q)
#pragma unroll
                    for (int b = 0; b < QB; ++b)
                        if (cs + lane + 32 * b < ccq[q]) red_add(gdst + rr[q][b], vv[q][b] * hq[q], pl);
            }
        }
    };

    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        const XT *gk = gbuf(k);
        XT *gn = gbuf(k + 1);
        // x_i of this iteration's columns (written by the previous iteration's
        // steps, published by the grid barrier)
        const double xi = mine ? ldcg_hint(a.x + c_i, pf) : 0.0;

        // ---------------- gradients, one column at a time; the next column's
        // row indices load while the current one is gathered
        closed = 0;
        grad = XT(0);
        {
            // Three register sets rotate over the columns: at step t the gathers
            // of column t+1 are issued, the entries of column t+2 are loaded,
            // then the products of column t (gathered one step earlier) are taken.
            struct Set {
                int32_t row[R][2];
                EV val[R][2], gv[R][2];
            };
            Set sa, sb, sc;
            auto cnt_of = [&](int t) { return t < T ? __shfl_sync(FULL, c_d.cnt, t) : 0; };
            auto load = [&](int t, Set &st) {
                if (t < T) load_runs(__shfl_sync(FULL, c_d.pbeg, t), cnt_of(t), st.row, st.val);
            };
            auto gather = [&](int t, Set &st) {
                if (t < T) gather_runs(gk, cnt_of(t), st.row, st.gv);
            };
            auto finish = [&](int t, const Set &st) {
                // the column kWarpAhead positions on goes to L2 now
                if (mine && lane == t + kWarpAhead) prefetch_col(c_d);
                const int cc = cnt_of(t);
                Part sum = dot_runs(cc, st.val, st.gv);
                if (cc > RUN * R) dot_tail(gk, __shfl_sync(FULL, c_d.pbeg, t), cc, sum);   // warp-uniform
                close_col(sum);
            };
            load(0, sa);
            gather(0, sa);
            load(1, sb);
            for (int t = 0; t < T; t += 3) {
                gather(t + 1, sb);
                load(t + 2, sc);
                finish(t, sa);
                if (t + 1 >= T) break;
                gather(t + 2, sc);
                load(t + 3, sa);
                finish(t + 1, sb);
                if (t + 2 >= T) break;
                gather(t + 3, sa);
                load(t + 4, sb);
                finish(t + 2, sc);
            }
        }

        // CERT: the zero steps the FP32 bound decides; the other columns in FP64
        bool certified = false;
        if constexpr (CERT) {
            certified = mine && a.problem == 0 && is_zero_bits(xi) && ZeroCert{own_s, own_a, own_m}.below(c_d.cnt + 5, lamf);
            fp64_grads(__ballot_sync(FULL, mine && !certified), gk);
        }

        // the sample of k+1 (integer work) and its descriptors
        {
            const SampleKey key = warp_sample_key(a.seed, k + 1, a.n);
            n_i = mine ? sample_index(uint32_t(j), key) : 0;
            n_d = c_d;   // (unused by the lanes without a position)
            if (mine) n_d = load_col(a.desc, n_i, pf);
        }

        // ---------------- the step of eq. (h(x)) (FP64) in the owner lanes
        XT h = XT(0);
        if (mine) {
            bool zero_step = certified;
            if constexpr (GM == 0) {
                if constexpr (sizeof(XT) == 4)
                    zero_step = a.problem == 0 && is_zero_bits(xi) && fabsf(float(grad)) <= lamf;
                else
                    zero_step = zero_step || (a.problem == 0 && is_zero_bits(xi) && abs_le_bits(double(grad), a.lambda));
            }
            if (!zero_step) {
                const double xn = coord_step(a.problem, xi, double(grad), double(c_d.invL), a.inv_beta, a.lambda, a.kappa);
                const double h64 = xn - xi;
                h = XT(h64);
                if (h64 != 0.0) {   // most steps are zero: x_i unchanged
                    st_hint(a.x + c_i, xn, pf);
                    cnt.nonzero += 1;
                    cnt.scattered += (unsigned long long)c_d.cnt;
                }
            }
            cnt.gathered += (unsigned long long)c_d.cnt;
        }

        // ---------------- scatter of the steps of k-1 and k into the other buffer
        scatter_owned(p_d, h_prev, gn);
        scatter_owned(c_d, h, gn);
        h_prev = h;
        p_d = c_d;
        // the next iteration's first columns go to L2 during the barrier
        if (it + 1 < iters && lane < kWarpAhead && mine) prefetch_col(n_d);

        // ---------------- the only grid barrier of the iteration
        const unsigned long long target = (unsigned long long)(it + 1) * gridDim.x;
        if (!grid_sync(a.bar, target, a.status, a.timeout_ns)) return;
        c_i = n_i;
        c_d = n_d;
    }
    // Both buffers equal again: the last iteration's steps go into the buffer
    // that holds g_{k0+iters-1}.
    if (iters > 0) scatter_owned(p_d, h_prev, gbuf(k0 + iters - 1));
    if (mine) sample_buf(a, k0 + iters)[j] = c_i;
    flush_counters(cnt, a.counters);
}

template <typename VT, typename XT>
int Kernels<VT, XT>::warp_max_blocks(int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    // the same grid serves every variant (gradient maps, certificate): the smallest co-resident grid
    const void *fns[3] = {(const void *)k_fused_warp<VT, XT, 0, false>, (const void *)k_fused_warp<VT, XT, 1, false>,
                          (const void *)k_fused_warp<VT, XT, 0, true>};
    const int nf = sizeof(XT) == 8 ? 3 : 2;
    int best = -1;
    for (int f = 0; f < nf; ++f) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[f], threads, 0) != cudaSuccess) return 0;
        if (best < 0 || per_sm < best) best = per_sm;
    }
    return best * sms;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::fused_warp(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                        bool zero_cert, cudaStream_t st)
{
    if (iters <= 0 || a.tau <= 0) return cudaSuccess;
    IterArgs<VT, XT> args = a;
    void *params[] = {(void *)&args, (void *)&k0, (void *)&iters};
    // the certificate applies to the FP64 form of LASSO
    const void *fn = a.problem == 2 ? (const void *)k_fused_warp<VT, XT, 1, false>
                     : (sizeof(XT) == 8 && zero_cert && a.problem == 0) ? (const void *)k_fused_warp<VT, XT, 0, true>
                                                                       : (const void *)k_fused_warp<VT, XT, 0, false>;
    return cudaLaunchCooperativeKernel(fn, dim3(unsigned(sh.blocks)), dim3(unsigned(sh.threads)), params, 0, st);
}

}  // namespace pcdm
