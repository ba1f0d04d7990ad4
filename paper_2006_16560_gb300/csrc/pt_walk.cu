// pt_walk.cu -- group-wise tree walk emitting the cell and particle-particle
// (PP) interaction lists of every group.
//
// One warp walks one group: it pops up to 32 nodes from a shared-memory
// stack, tests them in parallel and emits accepted cells, opened leaves'
// particles and opened internal nodes' children with warp prefix sums.  All
// tests are exact integer arithmetic on the grid boxes (see pt.h), so the
// lists are identical to the CPU oracle's.  A leaf opened for the opening
// angle alone (its box at least r_out from the group's box, so no pair can be
// within r_out) goes to the group's far PP segment, every other opened leaf
// to the near one; the force kernel skips the changeover test on the far
// segment.  Two ways to place the lists:
// - two passes: a counting pass sizes every group's lists, an exclusive scan
//   places them, and a filling pass writes them (both visit nodes in the
//   same order); used when no size estimate exists, and by batches;
// - one pass: each warp takes chunks of the list arrays from a bump
//   allocator and writes a group's lists contiguously into its chunk,
//   moving the group's entries so far to a fresh, larger chunk when the
//   current one fills.  Offsets are then in allocation order rather than
//   group order.  The arrays are sized from the previous walk of the tree;
//   if they run out, the kernel flags it and the host falls back to two
//   passes.
// Warps take groups from an atomic work counter (persistent grid).
#include "pt_kernels.cuh"

namespace pt {

constexpr int kWalkWarps = 4;
constexpr int kWalkThreads = 32 * kWalkWarps;


// Makes room for `need` entries of the current group in the one-pass list
// array: the group's entries so far ([g0, g0 + have)) move to a new chunk of
// max(chunk, 2 need) entries.  Returns false (and flags) when the array is full.
__device__ __forceinline__ bool grow_list(unsigned *arr, unsigned long long cap,
                                          unsigned long long *cursor, unsigned long long &g0,
                                          unsigned long long &end, unsigned have, unsigned long long need,
                                          unsigned long long chunk, unsigned *flags) {
    const unsigned lane = threadIdx.x & 31;
    unsigned long long size = 2 * need;
    if (size < chunk) size = chunk;
    unsigned long long nb = 0;
    if (lane == 0) nb = atomicAdd(cursor, size);
    nb = __shfl_sync(0xffffffffu, nb, 0);
    if (nb + size > cap) {
        if (lane == 0) atomicOr(flags, kErrListCap);
        return false;
    }
    __syncwarp();
    for (unsigned e = lane; e < have; e += 32) arr[nb + e] = arr[g0 + e];
    __syncwarp();
    g0 = nb;
    end = nb + size;
    return true;
}

template <bool FILL, bool MD, bool ONEPASS>
// 14 blocks per SM: the most the small stacks' shared memory allows (32 registers)
__global__ void __launch_bounds__(kWalkThreads, 14) k_walk(WalkArgs A) {
    extern __shared__ unsigned stack_mem[];      // kWalkWarps x A.stack_cap entries
    __shared__ long long ithr[kLevels];
    if (threadIdx.x < kLevels) ithr[threadIdx.x] = A.wp.ithr[threadIdx.x];
    __syncthreads();
    const unsigned w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned ng = A.st->ngroups;
    unsigned *stk = stack_mem + (size_t)w * A.stack_cap;
    const int cap = (int)A.stack_cap;
    // the bottom half of a full shared stack moves to the warp's spill area in
    // global memory and comes back when the shared part runs empty
    unsigned *gstk = A.spill + (size_t)(blockIdx.x * kWalkWarps + w) * A.spill_cap;
    const int half = cap / 2;            // >= 32 x 8, the most one step can push
    int max_sp = 0;
    // one pass: the warp's current chunks [.., c_end), [.., p_end) (near PP)
    // and [.., f_end) (far PP) and their first free entries (uniform across
    // the warp)
    unsigned long long c_free = 0, c_end = 0, p_free = 0, p_end = 0, f_free = 0, f_end = 0;
    bool dead = false;          // list array exhausted: keep walking, write nothing
    for (;;) {
        unsigned g = 0;
        if (lane == 0) g = atomicAdd(&A.st->work[FILL ? 1 : 0], 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const uint4 ga = A.gr_a[g], gb = A.gr_b[g];
        const long long r2thr = MD ? A.gr_thr[g] : A.sets[ga.w].r2thr;
        const int glo[3] = {2 * (int)ga.x, 2 * (int)ga.y, 2 * (int)ga.z};
        const int ghi[3] = {2 * (int)gb.x + 2, 2 * (int)gb.y + 2, 2 * (int)gb.z + 2};
        unsigned long long cbase = 0, pbase = 0, fbase = 0;
        if (ONEPASS) {
            cbase = c_free;
            pbase = p_free;
            fbase = f_free;
        } else if (FILL) {
            // the counting pass left the total PP count in gr_np: the group's
            // segment holds the near entries, then the far ones
            cbase = A.gr_co[g];
            pbase = A.gr_po[g];
            fbase = pbase + (A.gr_np[g] - A.gr_nf[g]);
        }
        unsigned nc = 0, nn = 0, nf = 0;
        if (lane == 0) stk[0] = gb.w;      // root of the group's set
        __syncwarp();
        int sp = 1;
        bool overflow = false;
        // a walk visits each node at most once; the cap only guards against a
        // corrupted tree turning into an endless loop
        unsigned iters = 0;
        int gsp = 0;
        while (sp > 0 || gsp > 0) {
            if (++iters > kWalkMaxIters) {
                overflow = true;
                break;
            }
            if (sp == 0) {               // refill from the spill area (its newest entries)
                const int r = gsp < half ? gsp : half;
                for (int e = lane; e < r; e += 32) stk[e] = gstk[gsp - r + e];
                gsp -= r;
                sp = r;
                __syncwarp();
            }
            const int k = sp < 32 ? sp : 32;
            sp -= k;
            const bool valid = (int)lane < k;
            const unsigned v = valid ? stk[sp + lane] : 0u;
            __syncwarp();
            bool accept = false, leaf = false, pfar = false;
            unsigned nch = 0, first = 0, pcount = 0, pbegin = 0;
            if (valid) {
                const uint4 a = A.nd_a[v], b = A.nd_b[v];
                const unsigned level = meta_level(a.w);
                const int sh = kBits - (int)level;
                const unsigned qmn[3] = {a.x, a.y, a.z}, qmx[3] = {b.x, b.y, b.z};
                long long d2 = 0, gap2 = 0;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const int p = (int)(qmn[d] >> sh);
                    const int c2 = (2 * p + 1) << sh;          // cube centre, half cells
                    int dd = glo[d] - c2;
                    dd = max(dd, c2 - ghi[d]);
                    dd = max(dd, 0);
                    d2 += (long long)dd * dd;
                    int gg = (int)qmn[d] - (ghi[d] >> 1);      // C.qmin - (G.qmax + 1)
                    gg = max(gg, (glo[d] >> 1) - (int)qmx[d] - 1);
                    gg = max(gg, 0);
                    gap2 += (long long)gg * gg;
                }
                // mass-dependent radii: the larger of the group's and the cell's threshold
                const long long thr = MD ? max(r2thr, A.nd_thr[v]) : r2thr;
                accept = (d2 >= ithr[level]) && (gap2 >= thr);
                leaf = meta_leaf(a.w);
                if (!accept) {
                    if (leaf) {
                        const uint2 r = A.nd_r[v];
                        pbegin = r.x;
                        pcount = r.y;
                        pfar = gap2 >= thr;      // opened for the opening angle only
                    } else {
                        nch = meta_nchild(a.w);
                        first = b.w;
                    }
                }
            }
            // accepted cells
            const unsigned amask = __ballot_sync(0xffffffffu, accept);
            if (ONEPASS && amask && !dead && cbase + nc + __popc(amask) > c_end)
                dead = !grow_list(A.cells, A.cap_cells, &A.st->work[0], cbase, c_end, nc,
                                  nc + __popc(amask), A.chunk_cells, &A.st->flags);
            if (FILL && accept && !dead) {
                unsigned long long pos = cbase + nc + __popc(amask & lanemask_lt());
                if (pos < A.cap_cells) A.cells[pos] = v;
                else atomicOr(&A.st->flags, kErrListCap);
            }
            nc += __popc(amask);
            // particles of opened leaves (near and far) and children of opened
            // internal nodes: one scan of the three counts in 11-, 11- and
            // 10-bit fields (warp sums below 2^11 when no leaf holds more
            // than 63 particles), else three scans
            const unsigned pn = pfar ? 0u : pcount, pf = pfar ? pcount : 0u;
            unsigned nincl, ntot, fincl, ftot, cincl, ctot;
            if (__any_sync(0xffffffffu, pcount > 63u)) {
                nincl = warp_incl_scan(pn);
                ntot = __shfl_sync(0xffffffffu, nincl, 31);
                fincl = warp_incl_scan(pf);
                ftot = __shfl_sync(0xffffffffu, fincl, 31);
                cincl = warp_incl_scan(nch);
                ctot = __shfl_sync(0xffffffffu, cincl, 31);
            } else {
                const unsigned all = warp_incl_scan(pn | (pf << 11) | (nch << 22));
                const unsigned tot = __shfl_sync(0xffffffffu, all, 31);
                nincl = all & 0x7ffu;
                fincl = (all >> 11) & 0x7ffu;
                cincl = all >> 22;
                ntot = tot & 0x7ffu;
                ftot = (tot >> 11) & 0x7ffu;
                ctot = tot >> 22;
            }
            if (ONEPASS && ntot && !dead && pbase + nn + ntot > p_end)
                dead = !grow_list(A.pp, A.cap_pp, &A.st->work[3], pbase, p_end, nn, nn + ntot,
                                  A.chunk_pp, &A.st->flags);
            if (ONEPASS && ftot && !dead && fbase + nf + ftot > f_end)
                dead = !grow_list(A.pp, A.cap_pp, &A.st->work[3], fbase, f_end, nf, nf + ftot,
                                  A.chunk_pp, &A.st->flags);
            if (FILL && (ntot | ftot) && !dead) {
                // every lane writes its own leaf's particle range at its offset
                const unsigned long long at = pfar ? fbase + nf + (fincl - pf) : pbase + nn + (nincl - pn);
                if (at + pcount <= A.cap_pp) {
                    for (unsigned e = 0; e < pcount; e++) A.pp[at + e] = pbegin + e;
                } else if (pcount) {
                    atomicOr(&A.st->flags, kErrListCap);
                }
            }
            nn += ntot;
            nf += ftot;
            if (sp + (int)ctot > cap) {
                if (gsp + half > (int)A.spill_cap) {
                    overflow = true;
                    break;
                }
                for (int e = lane; e < half; e += 32) gstk[gsp + e] = stk[e];
                __syncwarp();
                // shift the top part down by `half`, 32 entries at a time in
                // ascending order (each chunk is read before anything overlaps it)
                for (int e0 = half; e0 < sp; e0 += 32) {
                    const int e = e0 + (int)lane;
                    const unsigned x = e < sp ? stk[e] : 0u;
                    __syncwarp();
                    if (e < sp) stk[e - half] = x;
                    __syncwarp();
                }
                gsp += half;
                sp -= half;
            }
            for (unsigned j = 0; j < nch; j++) stk[sp + (cincl - nch) + j] = first + j;
            sp += (int)ctot;
            max_sp = max(max_sp, sp);
            __syncwarp();
        }
        if (overflow && lane == 0) atomicOr(&A.st->flags, kErrStack);
        if ((!FILL || ONEPASS) && lane == 0) atomicMax(&A.st->max_stack, (unsigned)max_sp);
        if (lane == 0) {
            if (!FILL) {                 // counting pass: gr_np holds the total for the scan
                A.gr_nc[g] = nc;
                A.gr_np[g] = nn + nf;
                A.gr_nf[g] = nf;
            } else {
                A.gr_np[g] = nn;
                A.gr_nf[g] = nf;
                A.gr_fo[g] = fbase;
                if (ONEPASS) A.gr_nc[g] = nc;
            }
        }
        if (ONEPASS) {
            if (lane == 0) {
                A.gr_co[g] = cbase;
                A.gr_po[g] = pbase;
                atomicAdd(&A.st->cell_total, (unsigned long long)nc);
                atomicAdd(&A.st->pp_total, (unsigned long long)(nn + nf));
            }
            c_free = cbase + nc;
            p_free = pbase + nn;
            f_free = fbase + nf;
        }
        __syncwarp();
    }
}

int walk_init() {
    // the largest stack the walk may use, set once per context (kernel
    // attributes are not stream work and stay out of captured graphs)
    const int smem = (int)((size_t)kWalkWarps * kWalkStackLarge * sizeof(unsigned));
    if (cudaFuncSetAttribute(k_walk<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_walk<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_walk<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_walk<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_walk<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_walk<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 1;
    return 0;
}

// The walk is latency bound: as many resident blocks as the stack allows.
static int walk_blocks(unsigned stack_cap) {
    const size_t smem = (size_t)kWalkWarps * stack_cap * sizeof(unsigned);
    int per_sm = (int)((200u * 1024u) / (smem + 2048));
    per_sm = per_sm < 1 ? 1 : (per_sm > 16 ? 16 : per_sm);   // 16 x 4 warps: the SM's limit
    return sm_count() * per_sm;
}

int walk_warps(unsigned stack_cap) { return walk_blocks(stack_cap) * kWalkWarps; }

int walk_launch(const WalkArgs &A, int phase, cudaStream_t st) {
    // work counters are reset by the caller (part of the status block)
    const size_t smem = (size_t)kWalkWarps * A.stack_cap * sizeof(unsigned);
    const int blocks = walk_blocks(A.stack_cap);
    if (phase == 2) {       // one pass (work[0] / work[3] are the list cursors)
        if (A.massdep) k_walk<true, true, true><<<blocks, kWalkThreads, smem, st>>>(A);
        else k_walk<true, false, true><<<blocks, kWalkThreads, smem, st>>>(A);
        return 1;
    }
    if (phase == 0) {
        if (A.massdep) k_walk<false, true, false><<<blocks, kWalkThreads, smem, st>>>(A);
        else k_walk<false, false, false><<<blocks, kWalkThreads, smem, st>>>(A);
        int nk = 1;
        nk += scan_exclusive<unsigned long long>(A.gr_nc, A.gr_co, &A.st->ngroups, &A.st->cell_total,
                                                 nullptr, A.scan_tmp, st);
        nk += scan_exclusive<unsigned long long>(A.gr_np, A.gr_po, &A.st->ngroups, &A.st->pp_total,
                                                 nullptr, A.scan_tmp, st);
        return nk;
    }
    if (A.massdep) k_walk<true, true, false><<<blocks, kWalkThreads, smem, st>>>(A);
    else k_walk<true, false, false><<<blocks, kWalkThreads, smem, st>>>(A);
    return 1;
}

}  // namespace pt
