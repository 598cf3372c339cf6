// Streaming persistent form of PCDM1 for long columns (Algorithm 1, step 4, the
// step of eq. (h(x)) with w = L).  Included at the end of pcdm_kernels.cuh.
//
// As in the pipelined kernel, one thread owns one sampled position per iteration
// (position j belongs to block j mod gridDim.x, thread j / gridDim.x), the
// residual is double-buffered (iteration k gathers from buffer k & 1 and adds the
// steps of iterations k-1 and k into the other one) and a single bounded grid
// barrier separates the iterations.  What differs is how the column reaches the
// thread: all of it, in chunks of kE entries, through two shared-memory slots of
// the thread, by TMA bulk copies (rows, then values) that complete on the
// thread's own mbarrier of the slot.  The copies run up to two chunks ahead of
// the gathers and continue into the next iteration's column, which is already
// known (the sample of k+1 is drawn during iteration k), so the column data never
// occupy the load/store pipe that the scattered gathers of g saturate; for a
// column of c entries the thread issues about c/kE pairs of bulk copies instead
// of 3c/4 (FP64) vector loads spread over 32 cache lines per warp instruction.
// The scatter of a moving coordinate (about 1% of LASSO's) rereads its column
// from memory.
#pragma once

namespace pcdm {

template <typename VT>
__host__ __device__ constexpr size_t stream_smem_bytes(int threads)
{
    // two slots per thread, then two mbarriers per thread
    return size_t(2) * size_t(threads) * size_t(pipe_slot_bytes<VT>()) + size_t(threads) * 16;
}

template <typename VT, typename XT, int GM = 0>
__global__ void __launch_bounds__(kPipeMaxBlock, 1) k_fused_stream(const IterArgs<VT, XT> a, int64_t k0,
                                                                   int64_t iters)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int VW = pipe_value_words<VT>();
    constexpr int SB = pipe_slot_bytes<VT>();
    constexpr int G = pad_granule<VT>();
    constexpr int EPW = 16 / int(sizeof(VT));
    const int nt = blockDim.x, t = threadIdx.x;
    const int64_t j0 = int64_t(t) * gridDim.x + blockIdx.x;
    const bool own = j0 < a.tau;
    uint64_t *mb = reinterpret_cast<uint64_t *>(smem + size_t(2) * nt * SB) + 2 * t;   // this thread's mbarriers
    Counters cnt;
    const uint64_t pf = l2_evict_first();   // A, descriptors, x
    const uint64_t pl = l2_evict_last();    // the residual buffers
    const float lamf = __double2float_rd(a.lambda);
    auto slot = [&](int s) { return smem + (size_t(s) * nt + t) * SB; };
    auto gbuf = [&](int64_t kk) { return (kk & 1) ? a.g2 : a.g; };
    auto chunks = [&](const Col<XT> &d) { return (d.cnt + kE - 1) / kE; };

    mbar_init(&mb[0], 1u);
    mbar_init(&mb[1], 1u);
    fence_mbarrier_init();
    __syncthreads();

    // The stream of this thread's copies: the chunks of the current column, then
    // those of the next one.  Item r goes to slot r & 1; it may be issued once
    // item r - 2 (the slot's previous content) has been read.
    int32_t i_cur = 0, i_nxt = 0;
    Col<XT> d_cur, d_nxt, d_prev;
    d_cur.pbeg = d_nxt.pbeg = d_prev.pbeg = 0;
    d_cur.cnt = d_nxt.cnt = d_prev.cnt = 0;
    d_cur.invL = d_nxt.invL = d_prev.invL = XT(0);
    if (own) {
        i_cur = ldcg(sample_buf(a, k0) + j0);
        d_cur = load_col(a.desc, i_cur, pf);
        i_nxt = sample_index(uint32_t(j0), make_sample_key(a.seed, k0 + 1, a.n));
        d_nxt = load_col(a.desc, i_nxt, pf);
    }
    int iss_c = 0, iss_n = 0;          // chunks of the current / next column issued
    uint32_t issued = 0, done = 0;     // items issued / read
    auto issue_one = [&]() -> bool {
        int64_t pbeg;
        int cnt_c, q;
        if (iss_c < chunks(d_cur)) {
            pbeg = d_cur.pbeg;
            cnt_c = d_cur.cnt;
            q = iss_c++;
        } else if (iss_n < chunks(d_nxt)) {
            pbeg = d_nxt.pbeg;
            cnt_c = d_nxt.cnt;
            q = iss_n++;
        } else {
            return false;
        }
        const int s = int(issued & 1u);
        const int64_t pc = (int64_t(cnt_c) + G - 1) / G * G;
        const int64_t left = pc - int64_t(q) * kE;
        const uint32_t e = uint32_t(left < kE ? left : kE);
        const uint32_t br = e * 4u, bv = e * uint32_t(sizeof(VT));
        fence_proxy_async_shared();   // this thread's reads of the slot come before the copy into it
        mbar_arrive_expect_tx(&mb[s], br + bv);
        bulk_copy_g2s(slot(s), a.prow + pbeg + int64_t(q) * kE, br, &mb[s], pf);
        bulk_copy_g2s(slot(s) + 64, a.pval + pbeg + int64_t(q) * kE, bv, &mb[s], pf);
        issued += 1u;
        return true;
    };
    auto refill = [&]() {
        while (issued < done + 2u && issue_one()) {
        }
    };
    // Waits for the copies still in flight (before the block leaves).
    auto drain = [&]() {
        while (done < issued) {
            mbar_wait_bounded(&mb[done & 1u], (done >> 1) & 1u, a.status, a.timeout_ns);
            done += 1u;
        }
    };
    if (own) refill();

    XT h_prev = XT(0);
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        const XT *gk = gbuf(k);
        XT *gn = gbuf(k + 1);
        XT h = XT(0);
        double xi = 0.0;
        bool need_step = false;
        double step_grad = 0.0;
        int32_t i_nn = 0;
        Col<XT> d_nn = d_nxt;
        const int valid = own ? d_cur.cnt : 0;
        bool ok = true;
        if (own) {
            xi = ldcg_hint(a.x + i_cur, pf);
            XT acc = XT(0);
            const int nc = chunks(d_cur);
            // Chunk q: wait for its copy, read its rows and values into registers,
            // free the slot (the copy two items ahead may start), gather g at its rows.
            auto load_gather = [&](int q, XT (&val)[kE], XT (&gv)[kE]) -> bool {
                if (!mbar_wait_bounded(&mb[done & 1u], (done >> 1) & 1u, a.status, a.timeout_ns)) return false;
                const unsigned char *sl = slot(int(done & 1u));
                int32_t row[kE];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const uint4 r4 = reinterpret_cast<const uint4 *>(sl)[w];
                    row[4 * w + 0] = int32_t(r4.x);
                    row[4 * w + 1] = int32_t(r4.y);
                    row[4 * w + 2] = int32_t(r4.z);
                    row[4 * w + 3] = int32_t(r4.w);
                }
#pragma unroll
                for (int w = 0; w < VW; ++w) {
                    XT vw[EPW];
                    decode_word<VT, XT>(reinterpret_cast<const uint4 *>(sl + 64)[w], vw);
#pragma unroll
                    for (int e = 0; e < EPW; ++e) val[w * EPW + e] = vw[e];
                }
                done += 1u;
                refill();
                const int v = valid - q * kE;
#pragma unroll
                for (int e = 0; e < kE; ++e) gv[e] = (e < v) ? ldcg_hint(gk + row[e], pl) : XT(0);
                return true;
            };
            auto dot = [&](int q, const XT (&val)[kE], const XT (&gv)[kE]) {
                const int v = valid - q * kE;
#pragma unroll
                for (int e = 0; e < kE; ++e)
                    if (e < v) acc = fma(val[e], grad_map<GM>(gv[e]), acc);
            };
            if constexpr (sizeof(XT) == 4) {
                // FP32 residual: the gathers of chunk q+1 are issued before the
                // products of chunk q, two chunks of values and gathers in registers
                XT va[kE], ga[kE], vb[kE], gb[kE];
                if (nc > 0) ok = load_gather(0, va, ga);
                if (ok) {
                    i_nn = sample_index(uint32_t(j0), make_sample_key(a.seed, k + 2, a.n));
                    d_nn = load_col(a.desc, i_nn, pf);
                }
                for (int q = 0; ok && q < nc; q += 2) {
                    if (q + 1 < nc && !(ok = load_gather(q + 1, vb, gb))) break;
                    dot(q, va, ga);
                    if (q + 1 >= nc) break;
                    if (q + 2 < nc && !(ok = load_gather(q + 2, va, ga))) break;
                    dot(q + 1, vb, gb);
                }
            } else {
                // FP64: one chunk at a time (two chunks of FP64 values and gathers
                // would not fit the registers of a 448-thread block)
                XT val[kE], gv[kE];
                for (int q = 0; q < nc; ++q) {
                    if (!(ok = load_gather(q, val, gv))) break;
                    if (q == 0) {
                        // the sample of k+2 (integer work) while the first gathers are in flight
                        i_nn = sample_index(uint32_t(j0), make_sample_key(a.seed, k + 2, a.n));
                        d_nn = load_col(a.desc, i_nn, pf);
                    }
                    dot(q, val, gv);
                }
            }
            if (nc == 0 && sizeof(XT) != 4) {
                i_nn = sample_index(uint32_t(j0), make_sample_key(a.seed, k + 2, a.n));
                d_nn = load_col(a.desc, i_nn, pf);
            }
            bool zero_step = false;
            if constexpr (GM == 0) {
                if constexpr (sizeof(XT) == 4)
                    zero_step = a.problem == 0 && is_zero_bits(xi) && fabsf(float(acc)) <= lamf;
                else
                    zero_step = a.problem == 0 && is_zero_bits(xi) && abs_le_bits(double(acc), a.lambda);
            }
            if (!zero_step) {
                need_step = true;
                step_grad = double(acc);
            }
            cnt.gathered += (unsigned long long)valid;
        }
        // a copy that never completed: the block leaves (the host reports the timeout)
        if (__syncthreads_or(ok ? 0 : 1)) {
            drain();
            return;
        }

        // ---------------- the step of eq. (h(x)) (FP64), x_i and the counters
        if (need_step) {
            const double xn = coord_step(a.problem, xi, step_grad, double(d_cur.invL), a.inv_beta, a.lambda, a.kappa);
            const double h64 = xn - xi;
            h = XT(h64);
            if (h64 != 0.0) {   // most steps are zero: x_i unchanged
                st_hint(a.x + i_cur, xn, pf);
                cnt.nonzero += 1;
                cnt.scattered += (unsigned long long)valid;
            }
        }

        // ---------------- scatter of the steps of k-1 and k into the other buffer
        if (own && !is_zero_bits(h_prev)) mem_scatter<VT, XT>(a, d_prev, h_prev, gn, pf, pl);
        if (own && !is_zero_bits(h)) mem_scatter<VT, XT>(a, d_cur, h, gn, pf, pl);
        h_prev = h;
        d_prev = d_cur;

        // ---------------- the only grid barrier of the iteration
        const unsigned long long target = (unsigned long long)(it + 1) * gridDim.x;
        grid_arrive(a.bar);
        if (!grid_wait(a.bar, target, a.status, a.timeout_ns)) {
            drain();
            return;
        }
        i_cur = i_nxt;
        d_cur = d_nxt;
        iss_c = iss_n;
        i_nxt = i_nn;
        d_nxt = d_nn;
        iss_n = 0;
        if (own) refill();
    }
    // Both buffers equal again: the last iteration's steps go into the buffer
    // that holds g_{k0+iters-1}.
    if (iters > 0 && own && !is_zero_bits(h_prev))
        mem_scatter<VT, XT>(a, d_prev, h_prev, gbuf(k0 + iters - 1), pf, pl);
    drain();   // the copies of the next launch's first column land before the block leaves
    if (own) sample_buf(a, k0 + iters)[j0] = i_cur;
    flush_counters(cnt, a.counters);
}

template <typename VT, typename XT>
int Kernels<VT, XT>::stream_max_blocks(int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const size_t bytes = stream_smem_bytes<VT>(threads);
    const void *fns[2] = {(const void *)k_fused_stream<VT, XT, 0>, (const void *)k_fused_stream<VT, XT, 1>};
    int best = -1;
    for (int f = 0; f < 2; ++f) {
        if (cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[f], threads, bytes) != cudaSuccess) return 0;
        if (best < 0 || per_sm < best) best = per_sm;
    }
    return best * sms;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::fused_stream(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                          cudaStream_t st)
{
    if (iters <= 0 || a.tau <= 0) return cudaSuccess;
    IterArgs<VT, XT> args = a;
    void *params[] = {(void *)&args, (void *)&k0, (void *)&iters};
    const void *fn = a.problem == 2 ? (const void *)k_fused_stream<VT, XT, 1> : (const void *)k_fused_stream<VT, XT, 0>;
    return cudaLaunchCooperativeKernel(fn, dim3(unsigned(sh.blocks)), dim3(unsigned(sh.threads)), params,
                                       stream_smem_bytes<VT>(sh.threads), st);
}

}  // namespace pcdm
