// common.cuh -- device pieces shared by the cell-scan path (ecmc.cu) and the
// constraint-graph path (graph.cu) of libecmc: owner-word encoding, chain
// states, counters, bit-level FP64 order, union-find of conflict components,
// block scans and the bounded grid barrier of the persistent kernels.
// Everything lives in an unnamed namespace: each translation unit keeps its
// own copy.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ecmc.h"

namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr uint32_t NONE = 0xFFFFFFFFu;
// owner word of a disk (the paper's tag, Sec. 2.3): static, or active / stalled
// for chain c in the low 30 bits
constexpr uint32_t OWN_STATIC = 0u;
constexpr uint32_t OWN_ACTIVE = 0x40000000u;
constexpr uint32_t OWN_STALLED = 0x80000000u;
constexpr uint32_t OWN_CHAIN = 0x3FFFFFFFu;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr unsigned long long INF_BITS = 0x7FF0000000000000ull;  // +inf

constexpr int ST_RUNNING = 0, ST_STALLED = 1, ST_BLOCKED = 2;

// per-leg counters (reset at every leg start)
enum { LC_BLOCKED = 0, LC_LIFTS, LC_HORIZON, LC_ERR_CAP, LC_ERR_REC, LC_ORDER, LC_OWNER_FAIL,
       LC_CONTINUED,
       LC_P1LIFTS, LC_REPAIRED, LC_WBLOCKED, LC_CWINDOWS, LC_RESTARTS, LC_WEAK,
       LC_ROWWIN,  // claim windows run by the row pass (cell scan)
       LC_WWEAK,   // chains whose claim sets met on a weak claim, this window
       LC_BADXY, LC_BADID,  // inputs out of range (creation only)
       LC_N };
enum { CTL_NCOMP = 0, CTL_WORK, CTL_NABORT, CTL_NMEMB, CTL_N };
// cumulative counters
enum { TC_LIFTS = 0, TC_LEGS, TC_CONFLICT_LEGS, TC_REPAIRED, TC_HORIZON, TC_ORDER,
       TC_LOG_N, TC_N };

// Event records of repair rounds carry seq = round << 24 | count; those of a
// window's parallel pass have seq < 2^24.
constexpr uint32_t REPAIR_SEQ0 = 1u << 24;

// Bound on every grid-barrier wait of the persistent kernels.
constexpr unsigned long long BARRIER_TIMEOUT_NS = 60ull * 1000 * 1000 * 1000;

// Non-negative doubles (and +inf) order like their bit patterns; comparisons
// of such values run on the integer pipe.
__device__ __forceinline__ unsigned long long dbits(double v) {
    return (unsigned long long)__double_as_longlong(v);
}
// v < 0 for a value that is not -0.0 (subtractions of finite doubles never give -0.0)
__device__ __forceinline__ bool dneg(double v) {
    return __double_as_longlong(v) < 0 && dbits(v) != 0x8000000000000000ull;
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int o) {
    return (unsigned long long)__shfl_xor_sync(FULL, (long long)v, o);
}

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long v, int src) {
    return (unsigned long long)__shfl_sync(FULL, (long long)v, src);
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void atomic_min_time(double *p, double v) {
    // times are >= 0: their IEEE bit patterns order like the values
    atomicMin((unsigned long long *)p, (unsigned long long)__double_as_longlong(v));
}

__device__ int uf_find(int32_t *p, int x) {
    for (;;) {
        const int px = ((volatile int32_t *)p)[x];
        if (px == x) return x;
        const int ppx = ((volatile int32_t *)p)[px];
        if (ppx != px) atomicCAS(p + x, px, ppx);  // path halving
        x = px;
    }
}

__device__ void uf_union(int32_t *p, int a, int b) {
    for (;;) {
        a = uf_find(p, a);
        b = uf_find(p, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(p + a, a, b) == a) return;  // larger root under smaller
    }
}

// Block-wide exclusive scan of one int per thread (blockDim.x a multiple of 32,
// at most 1024).
__device__ int block_exscan(int v, int *warp_tot, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        const int t = lane < nw ? warp_tot[lane] : 0;
        int u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, u, o);
            if (lane >= o) u += y;
        }
        if (lane < nw) warp_tot[lane] = u - t;
        if (lane == 31) *total = u;
    }
    __syncthreads();
    const int r = warp_tot[w] + x - v;
    __syncthreads();
    return r;
}

// Shared-memory working set of uf_block: four int arrays of UF_SMEM_CAP
// entries (union-find parents, counts, component roots, final flags).
constexpr int UF_SMEM_CAP = 2048;
constexpr size_t UF_SMEM_BYTES = 4 * UF_SMEM_CAP * sizeof(int32_t);

// Conflict components (one block). first: edges from the parallel pass
// (blocked chain -> holder of the claim it met); later rounds: edges from
// components that met another chain. Components holding a chain whose events
// are not final ("dirty") are listed for the repair with their members.
// reset_abort: clear the abort count here (the persistent kernels clear it
// elsewhere, after every block has read it).
// sm (UF_SMEM_BYTES of shared memory, or null): with k <= UF_SMEM_CAP the
// parents, counts, roots and flags live there during the phases (each phase
// then waits on shared instead of global memory) and are written back to
// s.uf, s.comp_of and s.fin at the end.
// Round 1 when every blocked chain makes a pair with its partner alone (the
// common case): blist[0 .. nblk) are the window's blocked chains, pcnt[c]
// the blocked chains naming c as partner. A pair {a, p} is a component when
// nobody names a (pcnt[a] = 0), only a names p (pcnt[p] = 1) and p is not
// blocked; a chain without a partner is a component alone. Then the result
// is the dense union-find's, written directly: identity for every chain in
// no component, the root (the smaller index) for the members, components in
// increasing root order, the blocked member first. Returns false (nothing
// written) otherwise. Either way pcnt is back to 0 for the chains listed.
template <class S>
__device__ bool uf_pairs(const S &s, const int32_t *blist, int32_t *pcnt, int nblk,
                         bool reset_abort, int32_t *sm) {
    const int k = s.k, tid = threadIdx.x, nt = blockDim.x;
    int a = -1, p = -1;
    bool simple = true;
    if (tid < nblk) {
        a = blist[tid];
        p = s.partner[a];
        if (p < 0 || p >= k) p = -1;
        const int pa = pcnt[a];
        const int pp = p >= 0 ? pcnt[p] : 1;
        const int sp = p >= 0 ? s.status[p] : ST_STALLED;
        simple = pa == 0 && (p < 0 || (pp == 1 && sp != ST_BLOCKED));
    }
    const bool ok = __syncthreads_and(simple) != 0;
    if (tid < nblk && p >= 0) pcnt[p] = 0;
    if (!ok) return false;
    for (int c = tid; c < k; c += nt) {
        s.uf[c] = c;
        s.comp_of[c] = c;
        s.fin[c] = 1;
        s.abort_to[c] = -1;
    }
    // the pairs by root: rank and offset among them
    int32_t *root_sm = sm, *size_sm = sm + 64;
    const int root = p >= 0 ? min(a, p) : a;
    if (tid < nblk) {
        root_sm[tid] = root;
        size_sm[tid] = p >= 0 ? 2 : 1;
    }
    __syncthreads();
    if (tid < nblk) {
        int rank = 0, off = 0, total = 0;
        for (int j = 0; j < nblk; ++j) {
            total += size_sm[j];
            if (root_sm[j] < root) {
                ++rank;
                off += size_sm[j];
            }
        }
        s.uf[a] = root;
        s.comp_of[a] = root;
        s.fin[a] = 0;
        s.comp_root[rank] = root;
        s.comp_off[rank] = off;
        s.comp_mem[off] = a;
        if (p >= 0) {
            s.uf[p] = root;
            s.comp_of[p] = root;
            s.fin[p] = 0;
            s.comp_mem[off + 1] = p;
        }
        if (rank == 0) {
            s.comp_off[nblk] = total;
            s.ctl[CTL_NCOMP] = nblk;
            s.ctl[CTL_NMEMB] = total;
            s.ctl[CTL_WORK] = 0;
            if (reset_abort) s.ctl[CTL_NABORT] = 0;
        }
    }
    __syncthreads();
    return true;
}

template <class S>
__device__ void uf_block(const S &s, int first, int *warp_tot, int *tot, bool reset_abort,
                         int32_t *sm = nullptr, const int32_t *blist = nullptr,
                         int32_t *pcnt = nullptr, int nblk = -1) {
    const int k = s.k, tid = threadIdx.x, nt = blockDim.x;
    if (first && blist && sm && nblk >= 1 && nblk <= 64 && nblk <= nt) {
        if (uf_pairs(s, blist, pcnt, nblk, reset_abort, sm)) return;
        __syncthreads();
    } else if (first && blist && pcnt) {
        // (the dense pass does not read the partner counts: back to 0)
        for (int q = tid; q < nblk && q < k; q += nt) {
            const int p = s.partner[blist[q]];
            if (p >= 0 && p < k) pcnt[p] = 0;
        }
    }
    const bool local = sm != nullptr && k <= UF_SMEM_CAP;
    int32_t *uf = local ? sm : s.uf;
    int32_t *cnt = local ? sm + UF_SMEM_CAP : s.comp_cnt;
    int32_t *cof = local ? sm + 2 * UF_SMEM_CAP : s.comp_of;
    int32_t *fin = local ? sm + 3 * UF_SMEM_CAP : s.fin;
    for (int c = tid; c < k; c += nt) {
        if (first) {
            uf[c] = c;
            fin[c] = s.status[c] != ST_BLOCKED;
            s.abort_to[c] = -1;
        } else if (local) {
            // (adoptions in the last round may have joined trees in s.uf)
            uf[c] = s.uf[c];
            fin[c] = s.fin[c];
        }
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        int other = -1;
        if (first) {
            if (s.status[c] == ST_BLOCKED) other = s.partner[c];
        } else {
            other = s.abort_to[c];
            s.abort_to[c] = -1;
        }
        if (other >= 0 && other < k) uf_union(uf, c, other);
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        cof[c] = uf_find(uf, c);
        cnt[c] = 0;
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt)
        if (!fin[c]) cnt[cof[c]] = -1;  // dirty root
    __syncthreads();
    for (int c = tid; c < k; c += nt)
        if (cnt[cof[c]] != 0) fin[c] = 0;
    __syncthreads();
    for (int c = tid; c < k; c += nt)
        if (cnt[c] == -1) cnt[c] = 0;
    __syncthreads();
    for (int c = tid; c < k; c += nt)
        if (!fin[c]) atomicAdd(cnt + cof[c], 1);
    __syncthreads();
    // chunked exclusive scans over roots: member offsets and component index
    const int chunk = (k + nt - 1) / nt;
    const int lo = min(k, tid * chunk), hi = min(k, lo + chunk);
    int sc = 0, sm_ = 0;
    for (int c = lo; c < hi; ++c) {
        const int n = cnt[c];
        sc += n;
        sm_ += n > 0;
    }
    int oc = block_exscan(sc, warp_tot, tot);
    int om = block_exscan(sm_, warp_tot, tot + 1);
    for (int c = lo; c < hi; ++c) {
        const int n = cnt[c];
        if (n > 0) {
            s.comp_root[om] = c;
            s.comp_off[om] = oc;
            cnt[c] = oc;  // becomes the write cursor
            oc += n;
            ++om;
        }
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt)
        if (!fin[c]) s.comp_mem[atomicAdd(cnt + cof[c], 1)] = c;
    if (local)
        for (int c = tid; c < k; c += nt) {
            s.uf[c] = uf[c];
            s.comp_of[c] = cof[c];
            s.fin[c] = fin[c];
        }
    if (tid == 0) {
        s.comp_off[tot[1]] = tot[0];
        s.ctl[CTL_NCOMP] = tot[1];
        s.ctl[CTL_NMEMB] = tot[0];
        s.ctl[CTL_WORK] = 0;
        if (reset_abort) s.ctl[CTL_NABORT] = 0;
    }
    __syncthreads();
}

// Grid barrier of a cooperative launch. bar[0] counts the arrivals of the
// launch (zeroed before it): a block's arrival number old gives its barrier's
// target, the next multiple of gridDim.x, and the block waits until the
// count reaches it -- the last block to arrive has nothing further to do. A
// wait longer than limit_ns records ECMC_ETIMEOUT in *err and gives up; the
// return value is false once *err is set, and the caller then returns (every
// block then stops at its next barrier, or gives up waiting for the blocks
// that stopped).
__device__ bool grid_sync(unsigned int *bar, int32_t *err, int *sflag,
                          unsigned long long limit_ns = BARRIER_TIMEOUT_NS) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int old = atomicAdd(bar, 1u);
        const unsigned int target = (old / gridDim.x + 1u) * gridDim.x;
        volatile unsigned int *cnt = bar;
        int ok = 1;
        if ((int)(*cnt - target) < 0) {
            const unsigned long long t0 = gtimer();
            while ((int)(*cnt - target) < 0) {
                if (gtimer() - t0 > limit_ns) {
                    ok = 0;
                    atomicExch(err, ECMC_ETIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *sflag = ok && *(volatile int32_t *)err == 0;
    }
    // (thread 0's fence after the wait orders the block's later loads: the
    // block barrier below passes that ordering on to its other threads)
    __syncthreads();
    return *sflag != 0;
}

}  // namespace
