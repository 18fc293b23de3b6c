// Beam-search kernel shared by the per-row-type translation units
// (search_f32.cu, search_bf16.cu, search_fp8.cu); host launch code lives in
// search.cu. See search.cu for the design.
#pragma once
#include "esg_internal.cuh"

namespace esg_sk {

constexpr int kBatch = 64;  // neighbours handled per expansion (R <= 64 per pass)

struct WarpSmem {
    uint32_t *hash;
    Cand *batch;
    uint32_t *nbuf;
    int *hcount;
};

__device__ __forceinline__ uint32_t hash_mix(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

// Visited set of one beam search: an open-addressing table in shared memory
// backed, once it reaches its load limit, by a larger table in a per-warp
// global-memory slot. visit() returns false iff `id` was already visited.
// Only when both tables are at their limits is an id reported as new without
// being stored (`saturated`; the list de-duplication then catches repeats).
// A global slot holds (tag << 32 | id), the tag being the work item's index
// + 1: a slot with another tag is free for this item, so the table is zeroed
// once per launch and never cleared between the items a warp runs. Its slots
// form buckets of 4 (one 32-byte sector); an id's probe sequence starts at
// the first slot of its bucket and runs on slot by slot, and slots are never
// freed within an item, so an id is either in its bucket or its bucket is full.
struct Visited {
    uint32_t *hs;   // shared table, hsize slots (a multiple of 4)
    uint32_t hsize;
    int *hcount;
    int hlimit;
    unsigned long long *hg;   // global overflow table, gmask + 1 slots
    uint32_t gmask;
    uint32_t tag;             // this item's tag (>= 1)
    int *gcount;
    int glimit;
    uint32_t *bm;             // per-warp shared bitmap of the buckets written in a pass (32 words)
};

__device__ __forceinline__ uint32_t global_bucket(const Visited &v, uint32_t id) {
    return hash_mix(id ^ 0x9e3779b9u) & (v.gmask >> 2);
}

// The shared table's slots form buckets of 4 (16 bytes). An id has two
// buckets, from two hashes by multiply-shift range reduction (any table
// size), and is stored in the one with more free slots, lowest free slot
// first, so a bucket's used slots are a prefix. An id is in one of its two
// buckets, or both were full when it came and it went to the global table:
// as slots are never freed within an item, an id found in neither bucket is
// new if either has a free slot, and looked up globally if both are full.
__device__ __forceinline__ void shared_buckets(const Visited &v, uint32_t id, uint32_t &b1, uint32_t &b2) {
    const uint32_t h = hash_mix(id);
    b1 = __umulhi(h, v.hsize >> 2);
    b2 = __umulhi(hash_mix(h ^ 0x5bd1e995u), v.hsize >> 2);
}

__device__ __forceinline__ unsigned free_slots(uint4 s4) {
    return (s4.x == ESG_NONE ? 1u : 0u) | (s4.y == ESG_NONE ? 2u : 0u) | (s4.z == ESG_NONE ? 4u : 0u) |
           (s4.w == ESG_NONE ? 8u : 0u);
}

__device__ __forceinline__ bool holds(uint4 s4, uint32_t id) {
    return s4.x == id || s4.y == id || s4.z == id || s4.w == id;
}

// Shared-table part of one lane's visit: 0 = visited, 1 = new (stored here),
// 2 = not here and both buckets are full or the table is at its limit
// (continue in the global table).
__device__ __forceinline__ int visit_shared(const Visited &v, uint32_t id) {
    uint32_t b1, b2;
    shared_buckets(v, id, b1, b2);
    const uint4 *h4 = reinterpret_cast<const uint4 *>(v.hs);
    for (;;) {
        const uint4 s1 = h4[b1], s2 = h4[b2];
        if (holds(s1, id) || holds(s2, id)) return 0;
        const unsigned f1 = free_slots(s1), f2 = free_slots(s2);
        if ((f1 | f2) == 0u || *(volatile int *)v.hcount >= v.hlimit) return 2;
        const bool first = __popc(f1) >= __popc(f2);
        const uint32_t slot = ((first ? b1 : b2) << 2) + (__ffs(first ? f1 : f2) - 1);
        const uint32_t prev = atomicCAS(&v.hs[slot], ESG_NONE, id);
        if (prev == ESG_NONE) { atomicAdd(v.hcount, 1); return 1; }
        if (prev == id) return 0;
    }
}

// Global-table visit by one lane, probing slot by slot from `start`: the
// swap resolves races between lanes. Returns true iff `id` is new.
__device__ __forceinline__ bool visit_global_from(const Visited &v, uint32_t id, uint32_t start, bool *saturated) {
    const unsigned long long mine = ((unsigned long long)v.tag << 32) | id;
    for (uint32_t probe = 0; probe <= v.gmask; ++probe) {
        const uint32_t slot = (start + probe) & v.gmask;
        const unsigned long long cur = *(volatile unsigned long long *)&v.hg[slot];
        if ((uint32_t)(cur >> 32) == v.tag) {   // taken by this item
            if ((uint32_t)cur == id) return false;
            continue;
        }
        if (*(volatile int *)v.gcount >= v.glimit) { *saturated = true; return true; }
        // only this warp's lanes write its table, always with this tag: a
        // failed swap leaves a slot of this item, holding `id` or another id
        const unsigned long long prev = atomicCAS(&v.hg[slot], cur, mine);
        if (prev == cur) { atomicAdd(v.gcount, 1); return true; }
        if (prev == mine) return false;
    }
    *saturated = true;
    return true;
}

// One lane's visit (the entry points). Returns true iff `id` is new.
__device__ __forceinline__ bool visit(const Visited &v, uint32_t id, bool *saturated) {
    const int r = visit_shared(v, id);
    if (r < 2) return r == 1;
    if (v.hg == nullptr) { *saturated = true; return true; }
    return visit_global_from(v, id, global_bucket(v, id) << 2, saturated);
}

// A loaded bucket (slots pa, pb) for `id`: whether it holds `id`, and the
// mask of its slots free for this item.
__device__ __forceinline__ void scan_bucket(const Visited &v, uint32_t id, ulonglong2 pa, ulonglong2 pb,
                                            bool &found, unsigned &freem) {
    const unsigned long long mine = ((unsigned long long)v.tag << 32) | id;
    const unsigned long long sl[4] = {pa.x, pa.y, pb.x, pb.y};
    found = false;
    freem = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        found |= sl[k] == mine;
        if ((uint32_t)(sl[k] >> 32) != v.tag) freem |= 1u << k;
    }
}

// One pass of the warp's global visits from bucket snapshots: `g` lanes have
// looked `id` up in bucket `b` (found, free slots); the lanes that insert
// into one bucket take its free slots in lane order (a second lane with the
// same id reports it visited) and store without a swap, since no other lane
// writes the table during the pass. Sets `n` (new) for `g` lanes; returns
// true where the bucket was full (the caller continues slot by slot).
__device__ __forceinline__ bool global_pass(const Visited &v, bool g, uint32_t id, uint32_t b, bool found,
                                            unsigned freem, bool &n, bool *saturated) {
    const int lane = threadIdx.x & 31;
    const unsigned long long mine = ((unsigned long long)v.tag << 32) | id;
    bool want = g && !found;
    if (g && found) n = false;
    if (want && *(volatile int *)v.gcount >= v.glimit) { *saturated = true; n = true; want = false; }
    const unsigned grp = __match_any_sync(0xffffffffu, want ? b : (0x80000000u | (unsigned)lane));
    bool dup = false;
    if (__any_sync(0xffffffffu, want && __popc(grp) > 1)) {
        const unsigned below = grp & ((1u << lane) - 1);
#pragma unroll 1
        for (int src = 0; src < 32; ++src) {
            const uint32_t oid = __shfl_sync(0xffffffffu, id, src);
            if (want && ((below >> src) & 1u) && oid == id) dup = true;
        }
    }
    const unsigned ins = __ballot_sync(0xffffffffu, want && !dup) & grp;
    bool full = false;
    if (want) {
        if (dup) {
            n = false;   // the lowest lane with this id stores it
        } else {
            const int k = __popc(ins & ((1u << lane) - 1));
            if (k < __popc(freem)) {
                unsigned f = freem;
                for (int t = 0; t < k; ++t) f &= f - 1;
                __stcg(v.hg + ((size_t)b << 2) + (__ffs(f) - 1), mine);
                atomicOr(&v.bm[(b >> 5) & 31], 1u << (b & 31));
                n = true;
            } else {
                full = true;
            }
        }
    }
    const int added = __popc(__ballot_sync(0xffffffffu, want && !dup && !full));
    if (lane == 0 && added) atomicAdd(v.gcount, added);
    return full;
}

// The global-table part of visit_pair for the lanes with g0 / g1 set.
__device__ __forceinline__ void visit_pair_global_body(const Visited &v, uint32_t v0, uint32_t v1, bool g0,
                                                       bool g1, bool &n0, bool &n1, bool *saturated) {
    const int lane = threadIdx.x & 31;
    const uint32_t b0 = g0 ? global_bucket(v, v0) : 0u, b1 = g1 ? global_bucket(v, v1) : 0u;
    const ulonglong2 *q0 = reinterpret_cast<const ulonglong2 *>(v.hg + ((size_t)b0 << 2));
    const ulonglong2 *q1 = reinterpret_cast<const ulonglong2 *>(v.hg + ((size_t)b1 << 2));
    bool fd0 = false, fd1 = false;
    unsigned fm0 = 0, fm1 = 0;
    {   // both buckets' loads in flight together
        ulonglong2 p0a{0, 0}, p0b{0, 0}, p1a{0, 0}, p1b{0, 0};
        if (g0) { p0a = __ldcg(q0); p0b = __ldcg(q0 + 1); }
        if (g1) { p1a = __ldcg(q1); p1b = __ldcg(q1 + 1); }
        if (g0) scan_bucket(v, v0, p0a, p0b, fd0, fm0);
        if (g1) scan_bucket(v, v1, p1a, p1b, fd1, fm1);
    }
    const bool f0 = global_pass(v, g0, v0, b0, fd0, fm0, n0, saturated);
    __syncwarp();
    if (g1 && ((v.bm[(b1 >> 5) & 31] >> (b1 & 31)) & 1u))
        scan_bucket(v, v1, __ldcg(q1), __ldcg(q1 + 1), fd1, fm1);
    const bool f1 = global_pass(v, g1, v1, b1, fd1, fm1, n1, saturated);
    __syncwarp();
    if (f0) n0 = visit_global_from(v, v0, (b0 + 1) << 2, saturated);
    if (f1) n1 = visit_global_from(v, v1, (b1 + 1) << 2, saturated);
    v.bm[lane] = 0u;
    __syncwarp();
}

// One try of a lane's shared-table visit from its two loaded buckets (s1,
// s2): found: visited; both full, or the table at its limit (`room` false):
// on to the global table (r = 2); else a swap into the lowest free slot of the
// bucket with more free slots: stored (new), or the same id stored there by
// another lane (visited), or another id took the slot (still pending: the
// caller loads the buckets again).
__device__ __forceinline__ void shared_try(const Visited &v, uint32_t id, uint32_t b1, uint32_t b2, uint4 s1,
                                           uint4 s2, bool room, bool &pend, int &r, bool &stored) {
    if (holds(s1, id) || holds(s2, id)) { r = 0; pend = false; return; }
    const unsigned f1 = free_slots(s1), f2 = free_slots(s2);
    if ((f1 | f2) == 0u || !room) { r = 2; pend = false; return; }
    const bool first = __popc(f1) >= __popc(f2);
    const uint32_t slot = ((first ? b1 : b2) << 2) + (__ffs(first ? f1 : f2) - 1);
    const uint32_t prev = atomicCAS(&v.hs[slot], ESG_NONE, id);
    if (prev == ESG_NONE) { r = 1; pend = false; stored = true; }
    else if (prev == id) { r = 0; pend = false; }
}

// Visits of the two neighbours v0, v1 of each lane (ESG_NONE: none). The
// shared table first: all four buckets of the two ids loaded together,
// inserts by swap (a lane whose slot another id took loads again). Then, for
// the ids that go on to the global table, both buckets are loaded at once,
// the v0 pass stores, the v1 lanes whose bucket the v0 pass wrote load it
// again, and the v1 pass stores; ids whose bucket was full probe on slot by
// slot with swaps. All lanes call it.
// Out-of-line copy of the global part for the FP32 kernels: inlined, its
// state competes for registers with the whole expansion loop, and those
// kernels spill more.
static __device__ __noinline__ void visit_pair_global_call(const Visited &v, uint32_t v0, uint32_t v1, bool g0,
                                                           bool g1, bool &n0, bool &n1, bool *saturated) {
    visit_pair_global_body(v, v0, v1, g0, g1, n0, n1, saturated);
}

template <bool OUTLINE>
__device__ __forceinline__ void visit_pair(const Visited &v, uint32_t v0, uint32_t v1, bool &n0, bool &n1,
                                           bool *saturated) {
    const int lane = threadIdx.x & 31;
    int r0 = 0, r1 = 0;
    {   // shared table: all four buckets of the two ids loaded together,
        // inserts by swap; a lane whose slot another id took loads again
        bool p0 = v0 != ESG_NONE, p1 = v1 != ESG_NONE;
        uint32_t a0 = 0, a1 = 0, c0 = 0, c1 = 0;
        if (p0) shared_buckets(v, v0, a0, a1);
        if (p1) shared_buckets(v, v1, c0, c1);
        const uint4 *h4 = reinterpret_cast<const uint4 *>(v.hs);
        while (__any_sync(0xffffffffu, p0 || p1)) {
            const bool room = *(volatile int *)v.hcount < v.hlimit;
            const uint4 z = make_uint4(0, 0, 0, 0);
            uint4 s0a = z, s0b = z, s1a = z, s1b = z;
            if (p0) { s0a = h4[a0]; s0b = h4[a1]; }
            if (p1) { s1a = h4[c0]; s1b = h4[c1]; }
            bool st0 = false, st1 = false;
            if (p0) shared_try(v, v0, a0, a1, s0a, s0b, room, p0, r0, st0);
            if (p1) shared_try(v, v1, c0, c1, s1a, s1b, room, p1, r1, st1);
            const int n_st = __popc(__ballot_sync(0xffffffffu, st0)) + __popc(__ballot_sync(0xffffffffu, st1));
            if (lane == 0 && n_st) *v.hcount += n_st;
            __syncwarp();
        }
    }
    n0 = r0 == 1;
    n1 = r1 == 1;
    const bool g0 = r0 == 2, g1 = r1 == 2;
    if (!__any_sync(0xffffffffu, g0 || g1)) return;
    if (v.hg == nullptr) {
        if (g0 || g1) *saturated = true;
        n0 |= g0;
        n1 |= g1;
        return;
    }
    if (OUTLINE) visit_pair_global_call(v, v0, v1, g0, g1, n0, n1, saturated);
    else visit_pair_global_body(v, v0, v1, g0, g1, n0, n1, saturated);
}


// Storage types of the traversal rows (esg_dtype): elements per 16-byte vector.
template <int ST> struct Store;
template <> struct Store<ESG_F32> { static constexpr int EPV = 4; };
template <> struct Store<ESG_BF16> { static constexpr int EPV = 8; };
template <> struct Store<ESG_FP8E4M3> { static constexpr int EPV = 16; };

// Accumulate the distance terms of one 16-byte vector of a row against the
// query slice qs[0..EPV) (FP32 accumulation; FP8 codes times the row scale).
template <int ST>
__device__ __forceinline__ float accum_vec(const uint4 &raw, const float *qs, float scale, int metric,
                                           float acc) {
    float x[Store<ST>::EPV];
    if (ST == ESG_F32) {
        x[0] = __uint_as_float(raw.x); x[1] = __uint_as_float(raw.y);
        x[2] = __uint_as_float(raw.z); x[3] = __uint_as_float(raw.w);
    } else if (ST == ESG_BF16) {
        const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            x[2 * t] = __uint_as_float(w4[t] << 16);
            x[2 * t + 1] = __uint_as_float(w4[t] & 0xFFFF0000u);
        }
    } else {
        const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w4[t] >> (16 * h)) & 0xFFFFu);
                __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
                float2 f = __half22float2(*reinterpret_cast<__half2 *>(&hr));
                x[4 * t + 2 * h] = f.x * scale;
                x[4 * t + 2 * h + 1] = f.y * scale;
            }
        }
    }
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
#pragma unroll
    for (int e = 0; e < Store<ST>::EPV; e += 4) {
        const float4 q = q4[e / 4];
        if (metric == ESG_L2SQ) {
            float a = q.x - x[e], b = q.y - x[e + 1], c = q.z - x[e + 2], d = q.w - x[e + 3];
            acc = fmaf(a, a, acc); acc = fmaf(b, b, acc); acc = fmaf(c, c, acc); acc = fmaf(d, d, acc);
        } else {
            acc = fmaf(q.x, x[e], acc); acc = fmaf(q.y, x[e + 1], acc);
            acc = fmaf(q.z, x[e + 2], acc); acc = fmaf(q.w, x[e + 3], acc);
        }
    }
    return acc;
}

// Distances from the query (FP32, staged in shared memory `qs`) to the rows
// listed in nbuf[0..m), written to batch[0..m). Rows are nvec 16-byte
// vectors; LPR lanes share a row, each loading VPL vectors, and the loads of
// U passes are all issued before any reduction.
template <int ST, int VPL>
__device__ __forceinline__ void eval_rows(const uint4 *__restrict__ Xv, const float *__restrict__ scale8,
                                          int nvec, int LPR, const float *qs, const uint32_t *nbuf,
                                          int m, Cand *batch, int metric) {
    constexpr int EPV = Store<ST>::EPV;
    const int lane = threadIdx.x & 31;
    const int s = lane & (LPR - 1);
    const int g = lane / LPR;
    const int rows_per_pass = 32 / LPR;
    // vectors in flight per lane scaled so that at most ~16 FP32-equivalent
    // vectors are decoded per pass (more would spill registers)
    constexpr int W = ST == ESG_F32 ? 1 : (ST == ESG_BF16 ? 2 : 4);
    constexpr int U0 = 16 / (VPL * W);
    constexpr int U = U0 < 1 ? 1 : (U0 > 8 ? 8 : U0);
    for (int base = 0; base < m; base += rows_per_pass * U) {
        uint4 xv[U][VPL];
        uint32_t id[U];
        float sc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int row = base + u * rows_per_pass + g;
            id[u] = row < m ? nbuf[row] : ESG_NONE;
            sc[u] = 1.f;
            if (id[u] != ESG_NONE) {
                const uint4 *p = Xv + (size_t)id[u] * nvec + s;
#pragma unroll
                for (int v = 0; v < VPL; ++v) xv[u][v] = __ldg(p + v * LPR);
                if (ST == ESG_FP8E4M3) sc[u] = __ldg(scale8 + id[u]);
            } else {
#pragma unroll
                for (int v = 0; v < VPL; ++v) xv[u][v] = make_uint4(0, 0, 0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float acc = 0.f;
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                acc = accum_vec<ST>(xv[u][v], qs + (s + v * LPR) * EPV, sc[u], metric, acc);
            acc = warp_sum_group(acc, LPR);
            const int row = base + u * rows_per_pass + g;
            if (s == 0 && row < m) batch[row] = Cand{metric == ESG_L2SQ ? acc : -acc, id[u]};
        }
    }
    __syncwarp();
}

// Exact FP32 distances of the rows in nbuf[0..m) (re-rank of candidates
// found with low-precision rows): 8 lanes per row.
__device__ __forceinline__ void eval_rows_fp32(const float *__restrict__ X, int d, const float *qs,
                                               const uint32_t *nbuf, int m, Cand *out, int metric) {
    const int lane = threadIdx.x & 31;
    const int s = lane & 7, g = lane >> 3;
    const int nv = d / 4;
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
    for (int base = 0; base < m; base += 4) {
        const int row = base + g;
        const uint32_t id = row < m ? nbuf[row] : ESG_NONE;
        float acc = 0.f;
        if (id != ESG_NONE) {
            const float4 *x4 = reinterpret_cast<const float4 *>(X + (size_t)id * d);
#pragma unroll 4
            for (int v = s; v < nv; v += 8) {
                const float4 x = __ldg(x4 + v), q = q4[v];
                if (metric == ESG_L2SQ) {
                    float a = q.x - x.x, b = q.y - x.y, c = q.z - x.z, e = q.w - x.w;
                    acc = fmaf(a, a, acc); acc = fmaf(b, b, acc); acc = fmaf(c, c, acc); acc = fmaf(e, e, acc);
                } else {
                    acc = fmaf(q.x, x.x, acc); acc = fmaf(q.y, x.y, acc);
                    acc = fmaf(q.z, x.z, acc); acc = fmaf(q.w, x.w, acc);
                }
            }
        }
        acc = warp_sum_group(acc, 8);
        if (s == 0 && row < m) out[row] = Cand{metric == ESG_L2SQ ? acc : -acc, id};
    }
    __syncwarp();
}

// Merge the sorted batch B[0..b) into the sorted list A[0..a) in place
// (capacity C; no item of B equals one of A). An item's final position is its
// index plus the number of items of the other sequence before it. The batch
// positions are found first, against the unchanged list, and parked in
// `pos` (b entries); the list items then move right, 32 at a time from the
// end down to the first batch item's position (items before it stay), every
// lane reading before any lane writes, so that no item is overwritten before
// it is read (a list item never moves left); last the batch items are
// written. Items whose position reaches C are dropped.
// Returns the new length min(a + b, C).
__device__ __forceinline__ int warp_merge_inplace(Cand *A, int a, const Cand *B, int b, uint32_t *pos,
                                                  int C) {
    const int lane = threadIdx.x & 31;
    for (int j = lane; j < b; j += 32) pos[j] = (uint32_t)(j + lower_rank(A, a, B[j]));
    __syncwarp();
    // list items before the first batch item's position do not move
    const int first = b > 0 ? (int)pos[0] : a;
    for (int i0 = ((a - 1) >> 5) << 5; i0 >= (first & ~31); i0 -= 32) {
        const int i = i0 + lane;
        Cand x;
        int p = C;
        if (i < a) {
            x = A[i];
            p = i + lower_rank(B, b, x);
        }
        __syncwarp();
        if (p < C) A[p] = x;
        __syncwarp();
    }
    for (int j = lane; j < b; j += 32)
        if (pos[j] < (uint32_t)C) A[pos[j]] = B[j];
    __syncwarp();
    return min(a + b, C);
}

// List state of one beam search.
struct ListState {
    int len;       // items in the list
    int qn;        // in-range items kept (<= ef)
    Cand qworst;   // the ef-th in-range item when qn == ef, else +inf
    int first;     // position of the best unexpanded item, -1 if none
};

// Cut the list after its ef-th in-range item (Q keeps the best ef; nothing
// behind it can be expanded or returned) and refresh |Q| and the worst of Q.
__device__ __forceinline__ void truncate_list(const Cand *list, ListState &st, int ef,
                                              uint32_t pl, uint32_t pr) {
    const int lane = threadIdx.x & 31;
    int seen = 0;
    st.qn = 0;
    st.qworst = Cand{INFINITY, ESG_NONE};
    st.first = -1;
    for (int base = 0; base < st.len; base += 32) {
        const int i = base + lane;
        const uint32_t raw = i < st.len ? list[i].id : ESG_NONE;
        const uint32_t id = raw & ESG_ID_MASK;
        const bool inr = i < st.len && id >= pl && id <= pr;
        const unsigned bal = __ballot_sync(0xffffffffu, inr);
        const unsigned unexp = __ballot_sync(0xffffffffu, i < st.len && !(raw & ESG_EXPANDED));
        const int c = __popc(bal);
        if (seen + c >= ef) {
            // position of the (ef - seen)-th set bit of bal
            const int need = ef - seen;
            unsigned b = bal;
            for (int t = 1; t < need; ++t) b &= b - 1;
            const int pos = base + __ffs(b) - 1;
            st.len = pos + 1;
            st.qn = ef;
            st.qworst = list[pos];
            const unsigned keep_unexp = unexp & (pos - base == 31 ? 0xffffffffu : ((1u << (pos - base + 1)) - 1));
            if (st.first < 0 && keep_unexp) st.first = base + __ffs(keep_unexp) - 1;
            return;
        }
        if (st.first < 0 && unexp) st.first = base + __ffs(unexp) - 1;
        seen += c;
    }
    st.qn = seen;
}

// Admitted candidates sit in batch[0..BB) (BB a multiple of 64 and a power
// of two; rejected slots hold +inf). Sort them and merge them into `list` in
// place (nbuf, BB entries, is scratch), then truncate. Batches of at most 16
// are ordered by counting ranks, of at most 32 sorted in registers. Returns
// false when nothing was admitted.
__device__ __forceinline__ bool admit_batch(Cand *batch, int BB, Cand *cbuf, Cand *list, uint32_t *nbuf,
                                            ListState &st, int ef, int C, uint32_t pl, uint32_t pr,
                                            int &status) {
    const int lane = threadIdx.x & 31;
    int b = 0;
    for (int c = 0; c < BB; c += 32) b += __popc(__ballot_sync(0xffffffffu, batch[c + lane].id != ESG_NONE));
    if (b == 0) return false;
    const Cand *B;
    if (b <= 32) {
        const unsigned below = (1u << lane) - 1;
        int o = 0;
        for (int c = 0; c < BB && o < b; c += 32) {
            const Cand x = batch[c + lane];
            const bool k = x.id != ESG_NONE;
            const unsigned bal = __ballot_sync(0xffffffffu, k);
            if (k) cbuf[o + __popc(bal & below)] = x;
            o += __popc(bal);
        }
        __syncwarp();
        float d = lane < b ? cbuf[lane].d : INFINITY;
        uint32_t id = lane < b ? cbuf[lane].id : ESG_NONE;
        __syncwarp();
        if (b <= 16) {
            // few candidates (the common case once the beam has settled):
            // each lane's rank among them by counting, cheaper than a sort
            // network over 32 lanes (ties, which visited ids rule out, by lane)
            int rank = 0;
#pragma unroll 4
            for (int j = 0; j < b; ++j) {
                const float dj = __shfl_sync(0xffffffffu, d, j);
                const uint32_t ij = __shfl_sync(0xffffffffu, id, j);
                rank += (cand_less(dj, ij, d, id) || (j < lane && cand_eq(Cand{dj, ij}, Cand{d, id}))) ? 1 : 0;
            }
            if (lane < b) cbuf[rank] = Cand{d, id};
        } else {
            warp_sort32_reg(d, id);
            cbuf[lane] = Cand{d, id};
        }
        __syncwarp();
        B = cbuf;
    } else {
        if (BB == 64) warp_sort64(batch);
        else warp_sort_pow2(batch, BB);
        B = batch;
    }
    const bool dropped = st.len + b > C;
    st.len = warp_merge_inplace(list, st.len, B, b, nbuf, C);
    truncate_list(list, st, ef, pl, pr);
    // items beyond the capacity only matter when the list did not reach its
    // ef-th in-range item within it (otherwise truncation drops them anyway)
    if (dropped && st.qn < ef) status |= ESG_Q_OVERFLOW;
    return true;
}

struct SearchArgs {
    const float *X;        // FP32 rows (re-rank, and traversal when st == F32)
    const uint4 *Xv;       // traversal rows (FP32, BF16 or FP8) as 16-byte vectors
    const float *scale8;   // FP8 per-row scales
    int rerank;
    const uint32_t *adj;
    const int64_t *row_off;  // first adj row of each graph level (rank p of level t: row row_off[t] + p)
    const int32_t *entries;
    const float *queries;
    const int64_t *qidx;   // optional: query row of an item (build: the inserted point)
    const esg_piece *pieces;
    const int32_t *kq;     // per-query k (validated), 0 = invalid; null = kconst
    int kconst;
    int qshift;            // query of item i = i >> qshift (2 pieces per query: 1)
    const int32_t *ef_q;       // per-query beam width (learned budget) or null
    const int32_t *maxexp_q;   // per-query expansion cap (0 = default) or null
    int64_t n;
    int64_t n_items;
    int d, nvec, LPR, R, E, metric;
    int ef, max_exp, k_max;
    int width;             // candidates expanded per iteration (1 = Algorithm 1 order)
    int BB;                // batch capacity: width * R rounded up to 64
    int H, C;              // per warp: table slots and list items of the widest beam
    int lpe;               // list items per unit of an item's beam width (>= 2)
    unsigned long long *ghash;  // global overflow visited tables, G slots per warp (zeroed), or null
    int G;
    unsigned long long *queue;  // atomic work counter
    const int32_t *order = nullptr;  // optional: the counter's k-th value runs item order[range[0] + k]
    const int32_t *range = nullptr;  // optional, device: [first, end) of this launch's part of order
    Cand *res;             // [n_items, k_max]
    int32_t *res_cnt;      // [n_items]
    int32_t *res_status;   // [n_items]
    int64_t *res_stats;    // [n_items, ESG_ITEM_STATS]
};

// MINB: resident blocks of 128 threads per SM the register allocation is
// sized for (4: up to 128 registers; 5: up to 96, instantiated only where
// that compiles without spills).
template <int ST, int VPL, int MINB = 4>
__global__ void __launch_bounds__(128, MINB)
search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const size_t qbytes = ((size_t)a.d * 4 + 15) & ~(size_t)15;
    const size_t per_warp = (size_t)a.H * 4 + (size_t)a.C * 8 + (size_t)a.BB * 12 + 32 * 8 +
                            16 + 128 + qbytes;
    unsigned char *base = smem_raw + per_warp * wib;
    WarpSmem w;
    size_t off = 0;
    w.batch = (Cand *)(base + off); off += (size_t)a.BB * 8;
    Cand *cbuf = (Cand *)(base + off); off += 32 * 8;
    w.nbuf = (uint32_t *)(base + off); off += (size_t)a.BB * 4;
    w.hcount = (int *)(base + off); off += 16;
    uint32_t *gbits = (uint32_t *)(base + off); off += 128;
    gbits[lane] = 0u;
    float *qs = (float *)(base + off); off += qbytes;
    const int gwarp = blockIdx.x * wpb + wib;
    // the arena of C list items and H table slots is split per item: the
    // list takes what the item's beam needs, the visited table the rest
    unsigned char *arena = base + off;
    Visited vis;
    vis.hcount = w.hcount;
    vis.hg = a.ghash ? a.ghash + (size_t)gwarp * a.G : nullptr;
    vis.gmask = (uint32_t)a.G - 1;
    vis.tag = 0;
    vis.gcount = w.hcount + 1;
    vis.glimit = a.G / 2;   // buckets of 4 slots at most half full on average
    vis.bm = gbits;

    const int64_t first = a.range ? (int64_t)a.range[0] : 0;
    const int64_t count = a.range ? (int64_t)a.range[1] - first : a.n_items;
    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = (int64_t)atomicAdd(a.queue, 1ULL);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= count) break;
        if (a.order) item = a.order[first + item];
        unsigned long long t_start;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
        const int64_t qi = item >> a.qshift;
        const esg_piece pc = a.pieces[item];
        const int kq = a.kq ? a.kq[qi] : a.kconst;
        int64_t n_exp = 0, n_eval = 0, n_oor = 0, n_rr = 0;
        int status = 0;
        if (pc.kind == ESG_PIECE_NONE || kq <= 0) {
            if (lane == 0) { a.res_cnt[item] = 0; a.res_status[item] = 0; }
            if (lane < 4) a.res_stats[item * ESG_ITEM_STATS + lane] = 0;
            if (lane == 0) { a.res_stats[item * ESG_ITEM_STATS + 4] = (int64_t)t_start; a.res_stats[item * ESG_ITEM_STATS + 5] = (int64_t)t_start; }
            continue;
        }
        const uint32_t pl = (uint32_t)pc.pl, pr = (uint32_t)pc.pr;
        const bool is_graph = pc.kind == ESG_PIECE_GRAPH;
        // low-precision scans keep ef candidates for the FP32 re-rank
        const bool do_rerank = ST != ESG_F32 && a.rerank;
        const int efq = a.ef_q ? a.ef_q[qi] : a.ef;
        const int ef = (is_graph || do_rerank) ? max(efq, kq) : kq;
        const int mxq = a.maxexp_q ? a.maxexp_q[qi] : 0;
        const int max_exp = mxq > 0 ? mxq : a.max_exp;

        // query in shared memory (FP32)
        {
            const int64_t qrow = a.qidx ? a.qidx[item] : qi;
            const float4 *q4 = reinterpret_cast<const float4 *>(a.queries + qrow * (int64_t)a.d);
            for (int v = lane; v < a.d / 4; v += 32) reinterpret_cast<float4 *>(qs)[v] = __ldg(q4 + v);
            __syncwarp();
        }
        ListState st{0, 0, Cand{INFINITY, ESG_NONE}, -1};
        // list capacity for this item's beam (as the plan sizes it for the
        // widest one), a multiple of 32; the table gets 2 slots per item freed
        const int cap = min(a.C, ((max(a.lpe * ef, 256) + 31) / 32) * 32);
        Cand *list = reinterpret_cast<Cand *>(arena);
        w.hash = reinterpret_cast<uint32_t *>(arena + (size_t)cap * 8);
        vis.hs = w.hash;
        vis.hsize = (uint32_t)(a.H + 2 * (a.C - cap));
        vis.hlimit = (int)(vis.hsize / 8) * 7;   // two-choice buckets stay short up to 7/8
        bool saturated = false;

        if (!is_graph) {
            // Leaf piece: exact scan of [pl, pr] (Algorithm 4, first branch).
            for (int64_t c0 = pl; c0 <= (int64_t)pr; c0 += kBatch) {
                const int m = (int)(((int64_t)pr - c0 + 1) < kBatch ? ((int64_t)pr - c0 + 1) : kBatch);
                for (int j = lane; j < m; j += 32) w.nbuf[j] = (uint32_t)(c0 + j);
                __syncwarp();
                eval_rows<ST, VPL>(a.Xv, a.scale8, a.nvec, a.LPR, qs, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                for (int j = lane; j < a.BB; j += 32) {
                    const bool keep = j < m && (st.qn < ef || cand_less(w.batch[j], st.qworst));
                    if (!keep) w.batch[j] = Cand{INFINITY, ESG_NONE};
                }
                __syncwarp();
                admit_batch(w.batch, a.BB, cbuf, list, w.nbuf, st, ef, cap, pl, pr, status);
            }
        } else {
            // Graph piece: Algorithm 1 with POST filtering to [pl, pr].
            {   // the table starts 16-byte aligned and holds a multiple of 4 slots
                uint4 *h4 = reinterpret_cast<uint4 *>(w.hash);
                for (uint32_t i = lane; i < vis.hsize / 4; i += 32)
                    h4[i] = make_uint4(ESG_NONE, ESG_NONE, ESG_NONE, ESG_NONE);
            }
            if (lane == 0) { w.hcount[0] = 0; w.hcount[1] = 0; }
            __syncwarp();
            vis.tag = (uint32_t)item + 1u;
            const uint32_t *adj = a.adj + (size_t)a.row_off[pc.depth] * a.R;
            // entry points: into P, and into Q when in range
            {
                uint32_t e = ESG_NONE;
                if (lane < a.E) {
                    const int32_t v = a.entries[(size_t)pc.heap * a.E + lane];
                    if (v >= 0 && v < a.n) e = (uint32_t)v;
                }
                const bool nw = e != ESG_NONE && visit(vis, e, &saturated);
                const unsigned bal = __ballot_sync(0xffffffffu, nw);
                if (nw) w.nbuf[__popc(bal & ((1u << lane) - 1))] = e;
                const int m = __popc(bal);
                __syncwarp();
                eval_rows<ST, VPL>(a.Xv, a.scale8, a.nvec, a.LPR, qs, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                for (int j = lane; j < a.BB; j += 32) {
                    if (j >= m) w.batch[j] = Cand{INFINITY, ESG_NONE};
                    else n_oor += (w.batch[j].id < pl || w.batch[j].id > pr);
                }
                __syncwarp();
                admit_batch(w.batch, a.BB, cbuf, list, w.nbuf, st, ef, cap, pl, pr, status);
            }
            // all items before `hint` are expanded
            int hint = st.first < 0 ? st.len : st.first;
            for (;;) {
                // the (up to) `width` best unexpanded candidates, ascending
                int sel[4];
                int nsel = 0;
                for (int b0 = hint & ~31; b0 < st.len && nsel < a.width; b0 += 32) {
                    const int i = b0 + lane;
                    const bool f = i >= hint && i < st.len && !(list[i].id & ESG_EXPANDED);
                    unsigned bal = __ballot_sync(0xffffffffu, f);
                    while (bal && nsel < a.width) { sel[nsel++] = b0 + __ffs(bal) - 1; bal &= bal - 1; }
                }
                if (nsel == 0) break;
                if (n_exp >= max_exp) { status |= ESG_Q_TRUNCATED; break; }
                uint32_t us[4];
                for (int t = 0; t < nsel; ++t) us[t] = list[sel[t]].id & ESG_ID_MASK;
                __syncwarp();
                // mark in-range ones expanded; drop out-of-range ones (they are
                // neither in Q nor in P once expanded), highest position first
                for (int t = nsel - 1; t >= 0; --t) {
                    const int pos = sel[t];
                    if (us[t] >= pl && us[t] <= pr) {
                        if (lane == 0) list[pos].id = us[t] | ESG_EXPANDED;
                        __syncwarp();
                        continue;
                    }
                    const int cnt = st.len - 1 - pos;
                    for (int b0 = 0; b0 < cnt; b0 += 32) {
                        const bool act = b0 + lane < cnt;
                        Cand nx;
                        if (act) nx = list[pos + b0 + lane + 1];
                        __syncwarp();
                        if (act) list[pos + b0 + lane] = nx;
                        __syncwarp();
                    }
                    st.len -= 1;
                }
                hint = sel[0];
                n_exp += nsel;
                // neighbours of the selected candidates, visited-tested, compacted
                int m = 0;
                for (int t = 0; t < nsel; ++t) {
                    const uint32_t *row = adj + (size_t)us[t] * a.R;
                    for (int c64 = 0; c64 < a.R; c64 += 64) {
                        uint32_t v0 = c64 + lane < a.R ? __ldg(row + c64 + lane) : ESG_NONE;
                        uint32_t v1 = c64 + lane + 32 < a.R ? __ldg(row + c64 + lane + 32) : ESG_NONE;
                        if (v0 >= (uint64_t)a.n) v0 = ESG_NONE;   // malformed imported graph: ignore
                        if (v1 >= (uint64_t)a.n) v1 = ESG_NONE;
                        bool n0, n1;
                        visit_pair<ST == ESG_F32>(vis, v0, v1, n0, n1, &saturated);
                        const unsigned b0 = __ballot_sync(0xffffffffu, n0);
                        const unsigned b1 = __ballot_sync(0xffffffffu, n1);
                        const int c0 = __popc(b0);
                        if (n0) w.nbuf[m + __popc(b0 & ((1u << lane) - 1))] = v0;
                        if (n1) w.nbuf[m + c0 + __popc(b1 & ((1u << lane) - 1))] = v1;
                        m += c0 + __popc(b1);
                    }
                }
                __syncwarp();
                if (m == 0) continue;
                eval_rows<ST, VPL>(a.Xv, a.scale8, a.nvec, a.LPR, qs, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                // Algorithm 1's admission test, then de-duplication against
                // the list (only needed once the visited set saturates)
                const bool sat = __any_sync(0xffffffffu, saturated);
                for (int j = lane; j < a.BB; j += 32) {
                    bool keep = false;
                    if (j < m) {
                        const Cand x = w.batch[j];
                        n_oor += (x.id < pl || x.id > pr);
                        keep = st.qn < ef || cand_less(x, st.qworst);
                        if (keep && sat) {
                            const int p = lower_rank(list, st.len, x);
                            if (p < st.len && cand_eq(list[p], x)) keep = false;
                        }
                    }
                    if (!keep) w.batch[j] = Cand{INFINITY, ESG_NONE};
                }
                __syncwarp();
                if (admit_batch(w.batch, a.BB, cbuf, list, w.nbuf, st, ef, cap, pl, pr, status))
                    hint = st.first < 0 ? st.len : st.first;
            }
            if (__any_sync(0xffffffffu, saturated)) status |= ESG_Q_OVERFLOW;
        }
        // FP32 re-rank of the final in-range candidates found on low-precision
        // rows, in place: the first ef in-range items are moved to the front
        // (an item never moves right, and each chunk is read before it is
        // written), their exact distances computed, then sorted (the list
        // holds at least 4 ef items, so the power-of-two sort fits)
        if (do_rerank && st.len > 0) {
            int cnt = 0;
            for (int b0 = 0; b0 < st.len && cnt < ef; b0 += 32) {
                const int i = b0 + lane;
                const uint32_t id = i < st.len ? (list[i].id & ESG_ID_MASK) : ESG_NONE;
                const bool inr = i < st.len && id >= pl && id <= pr;
                const unsigned bal = __ballot_sync(0xffffffffu, inr);
                const int pos = cnt + __popc(bal & ((1u << lane) - 1));
                __syncwarp();
                if (inr && pos < ef) list[pos] = Cand{0.f, id};
                __syncwarp();
                cnt += __popc(bal);
            }
            cnt = min(cnt, ef);
            for (int c0 = 0; c0 < cnt; c0 += kBatch) {
                const int m = min(kBatch, cnt - c0);
                for (int j = lane; j < m; j += 32) w.nbuf[j] = list[c0 + j].id;
                __syncwarp();
                eval_rows_fp32(a.X, a.d, qs, w.nbuf, m, list + c0, a.metric);
            }
            n_rr += cnt;
            const int P = next_pow2_int(max(cnt, 2));
            for (int j = cnt + lane; j < P; j += 32) list[j] = Cand{INFINITY, ESG_NONE};
            __syncwarp();
            warp_sort_pow2(list, P);
            st.len = cnt;
        }
        // emit the first min(k, |Q|) in-range items
        {
            int written = 0;
            Cand *out = a.res + item * (int64_t)a.k_max;
            for (int b0 = 0; b0 < st.len && written < kq; b0 += 32) {
                const int i = b0 + lane;
                const uint32_t id = i < st.len ? (list[i].id & ESG_ID_MASK) : ESG_NONE;
                const bool inr = i < st.len && id >= pl && id <= pr;
                const unsigned bal = __ballot_sync(0xffffffffu, inr);
                const int pos = written + __popc(bal & ((1u << lane) - 1));
                if (inr && pos < kq) out[pos] = Cand{list[i].d, id};
                written += __popc(bal);
            }
            written = min(written, kq);
            n_exp = __shfl_sync(0xffffffffu, n_exp, 0);
            for (int o = 16; o > 0; o >>= 1) n_oor += __shfl_xor_sync(0xffffffffu, n_oor, o);
            if (lane == 0) {
                a.res_cnt[item] = written;
                a.res_status[item] = status;
                unsigned long long t_end;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                int64_t *rs = a.res_stats + item * ESG_ITEM_STATS;
                rs[0] = n_exp;
                rs[1] = n_eval;
                rs[2] = n_oor;
                rs[3] = n_rr;
                rs[4] = (int64_t)t_start;
                rs[5] = (int64_t)t_end;
            }
        }
        __syncwarp();
    }
}

}  // namespace esg_sk

namespace esg_sk {
typedef void (*SearchFn)(SearchArgs);
// occ5: the variant compiled for 5 blocks per SM (nullptr where none exists)
SearchFn pick_f32(int vpl, bool occ5 = false);
SearchFn pick_bf16(int vpl, bool occ5 = false);
SearchFn pick_fp8(int vpl, bool occ5 = false);
}  // namespace esg_sk
