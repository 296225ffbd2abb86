// tc_count.cu -- steps 3-4 of the method on the device: intersect N+(u) with
// N+(v) for every oriented edge and reduce to the total and t(v).
//
// Paper: Sec. 3.2 (the common neighbours w of an oriented edge (u, v) each
// close one triangle), Alg. 2 Compute_Intersection / Reduce, Sec. 4.2.2
// (TwoSmall: one thread per pair; TwoLarge: CTA-cooperative intersection of
// long lists), and the small x large kernel proposed in Sec. 5 (walk the
// shorter list, search the longer one).
//
// Three kernels share the work that the partition (tc_build.cu) cut:
//   k_count_small : one thread per source row u with d+(u) <= small_max;
//                   sorted merge of N+(u) with each short N+(v).
//   k_count_warp  : one warp per work item of a pivot with d+(p) <= warp_max;
//                   N+(p) goes into a warp-private rank-id hash table and the
//                   lists of 32 partners q at a time are walked as one
//                   flattened sequence of 16-byte vectors.
//   k_count_cta   : one CTA per work item of a longer pivot list; the table
//                   (one segment of N+(p), a direct cell per rank id of its
//                   span, a bitmap or a hash) is shared by all warps of the
//                   CTA, which walk the partners' padded rank-id lists with
//                   G lanes per partner by list-length class.
// Every element w of N+(q) is probed in the table of N+(p).
//
// Per-vertex counts: triangle {p, q, w} with w in N+(p) and N+(q) is found
// exactly once.  w is a key of the pivot's table, so its count accumulates in
// the table slot and is flushed once per item; q gets one atomic per partner
// with a non-zero count; p one atomic per item.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <string>

#include "tc_internal.cuh"

namespace tc {

struct CountArgs {
    const int64_t* rpp;
    const int32_t* colp;
    const int32_t* dp;
    const int64_t* prp;
    const int32_t* pcol;
    const int2* pdesc;            // beside pcol: (first vector of the partner's colr row, its d+)
    const Item* items;
    const unsigned long long* n_items;
    unsigned long long items_cap;   // allocated items (n_items never exceeds it; clamped anyway)
    unsigned int* queue;
    unsigned long long* totals;   // [G] (batch) or [1]
    unsigned long long* t;        // per-vertex counts or nullptr
    unsigned long long* t_rank;   // with t: counts of table keys, indexed by rank id (added into t at the end)
    const int32_t* row_graph;     // batch: graph of each vertex, else nullptr
    const int32_t* colr;          // oriented lists in rank ids, row u at colr_row(rpp, u), padded with -1
    const int32_t* perm;          // rank id -> vertex id
    const int2* rspan;            // smallest and largest rank id of each oriented row
    int bitmap_bits;              // max span (rank ids) of a bitmap table; 0 = off
    int direct_span;              // max span of a direct cell table (32-bit cells up to half of it); 0 = off
    int u_ints;                   // ints of the table region of k_count_cta
    int64_t n;
    int shard, nshards;           // this launch covers shard `shard` of `nshards` equal parts of the work
    int cap;                      // keys per table segment
    int small_max;
    int small_lanes;              // threads per row of k_count_small (power of two, <= 32)
    int64_t colr_len, colp_len;   // entries allocated for colr and colp (debug bounds checks)
};

constexpr int kProbeHash = 1;
constexpr int kProbeBsearch = 2;

// Device check word of the count kernels: a bit is raised (and the bad step
// skipped) when a kernel meets a state its invariants exclude, instead of
// spinning or touching memory out of bounds.  Sticky per device until
// tc_check reads and clears it.
__device__ unsigned g_tc_device_error = 0u;

__device__ __forceinline__ void raise_error(unsigned bit) { atomicOr(&g_tc_device_error, bit); }

// Bounds and invariant checks of the TC_DEBUG build (-DTC_DEBUG=1): a failed
// check raises its bit of the check word and the guarded access is skipped.
// In the release build every check is the constant true.
#ifndef TC_DEBUG
#define TC_DEBUG 0
#endif
__device__ __forceinline__ bool dbg_ok(bool cond, unsigned bit) {
    if (TC_DEBUG && !cond) {
        raise_error(bit);
        return false;
    }
    return true;
}

__device__ __forceinline__ unsigned hslot(int x, int logS) {
    return ((unsigned)x * 0x9E3779B1u) >> (32 - logS);
}

// Zero-encoded open addressing for the rank-id tables: a slot holds x+1, 0 is
// empty, so a table whose slots are reset after use is all zeros again.  The
// tables hold at most a quarter of their slots, so an insert always meets an
// empty slot and a lookup of a missing key an empty slot too; both loops are
// nevertheless bounded by the table size: a probe sequence that has visited
// every slot (a table left dirty by an earlier item) gives up and raises
// TC_DEVERR_PROBE.
__device__ __forceinline__ void table_insert_z(int* keys, int logS, int x) {
    const unsigned mask = (1u << logS) - 1u;
    unsigned h = hslot(x, logS);
    for (unsigned step = 0; step <= mask; ++step) {
        if (atomicCAS(&keys[h], 0, x + 1) == 0) return;
        h = (h + 1u) & mask;
    }
    raise_error(TC_DEVERR_PROBE);
}

__device__ __forceinline__ int table_find_z(const int* keys, int logS, int x) {
    const unsigned mask = (1u << logS) - 1u;
    unsigned h = hslot(x, logS);
    for (unsigned step = 0; step <= mask; ++step) {
        const int k = keys[h];
        if (k == x + 1) return (int)h;
        if (k == 0) return -1;
        h = (h + 1u) & mask;
    }
    raise_error(TC_DEVERR_PROBE);
    return -1;
}

// slot of x in the sorted keys[0, len), or -1 (binary search)
__device__ __forceinline__ int table_find_sorted(const int* keys, int len, int x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < x) lo = mid + 1; else hi = mid;
    }
    return (lo < len && keys[lo] == x) ? lo : -1;
}

__device__ __forceinline__ int warp_incl_scan_i(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

#ifndef TC_CTA_VEC
#define TC_CTA_VEC 4
#endif
#ifndef TC_CTA_LANE_SHIFT
#define TC_CTA_LANE_SHIFT 5
#endif
constexpr int kVec = TC_CTA_VEC;  // 16-byte vector loads in flight per lane
// the next work item's descriptors are copied ahead with cp.async
#ifndef TC_CTA_ITEM_PREFETCH
#define TC_CTA_ITEM_PREFETCH 1
#endif


// ---------------------------------------------------------------------------
// CTA-table kernel (persistent; items from a global queue)
//
// The whole CTA shares one table per item.  The item's partners are taken
// kCtaPer * blockDim at a time, counting-sorted by list-length class in shared
// memory and cut into warp tasks of 32/G partners of one class with G lanes
// per partner (cta_partners); warps take tasks longest class first from a
// shared counter, and each lane walks its part of the partner's padded
// rank-id list (probe_list_padded).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_excl_scan_i(int v, int* sm, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int inc = warp_incl_scan_i(v);
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int t = lane < nw ? sm[lane] : 0;
        const int ti = warp_incl_scan_i(t);
        if (lane < nw) sm[lane] = ti - t;
        if (lane == 31) sm[32] = ti;
    }
    __syncthreads();
    const int r = sm[w] + inc - v;
    *total = sm[32];
    __syncthreads();
    return r;
}

// partners sorted per sub-chunk, per thread of the CTA kernel
#ifndef TC_CTA_PER
#define TC_CTA_PER 2
#endif
constexpr int kCtaPer = TC_CTA_PER;

// Per-CTA partner scratch: the partners of one sub-chunk, sorted by list
// length class (longest first), and the warp tasks cut from them.
constexpr int kClasses = 16;
struct CtaScratch {
    int64_t* qb;            // [pmax] list start of each sorted partner
    int* q;                 // [pmax]
    int* dq;                // [pmax]
    unsigned char* tcls;    // [pmax] class of each task
    int* ccnt;              // [kClasses] partners per class
    int* coff;              // [kClasses] first sorted position of each class
    int* toff;              // [kClasses] first task of each class
    int* misc;              // [4]: task counter, number of tasks
    int* scan;              // [33]
};

// Table of one pivot segment.  Hash: open addressing over rank ids (or vertex
// ids for the binary-search mode).  Bitmap: bit (x - lo) set for each key x,
// with a per-word prefix of set bits so that a hit's counter index is its
// ordinal among the keys.
constexpr int kModeHash = 0;
constexpr int kModeBitmap = 1;
constexpr int kModeBsearch = 2;
constexpr int kModeDirect = 3;   // one 16-bit cell per rank id of the span
constexpr int kModeDirect32 = 4; // one 32-bit cell per rank id, for spans up to direct_span / 2
// Direct cells: a key's cell holds a marker (top bit) plus its hits.  With
// per-vertex counts every probe inside the span is one shared atomic add whose
// returned old value carries the marker, so a probe needs no separate load;
// cells of rank ids that are not keys collect junk counts (at most one per
// partner of the item, below the marker) and the whole span is cleared after
// the item.  32-bit cells go one step further: a probe outside the span is
// clamped to one of 32 dummy cells past it (span + lane, never marked), so
// every probe is the same unpredicated atomic; the dummies collect junk
// counts too (fewer than the item's probes, far below the marker) and are
// cleared with the span.
constexpr unsigned kMark32 = 0x80000000u;
constexpr unsigned kMark16 = 0x8000u;

struct Table {
    const int* keys;
    int* cnts;
    int logS, len;
    const unsigned* bits;
    const unsigned short* pre;
    unsigned short* cell;  // direct mode
    unsigned* cell32;      // direct mode, 32-bit cells
    int lo, span;
    int xthr;              // walks of partitioned lists may stop at a batch whose lowest vector is below this
    int64_t llen;          // entries of the list array walked (debug checks)
    unsigned lim;          // span + lane: clamp of 32-bit direct probes
    unsigned sbase;        // shared-memory address of the cell array (direct modes)
    int ucap;              // ints of the table region (debug checks)
    int wmax;              // words of the bitmap (debug checks)
};

// Smallest y >= 1 with rank_level(y) >= L (0: none below 2^32).  From octave 3
// on every level is taken: level 8e + s first at y = (8 + s) << (e - 3).
__device__ __forceinline__ unsigned level_min_y(int L) {
    if (L <= 0) return 1u;
    if (L >= kRankLevels) return 0u;
    if (L >= 24) return (8u + (unsigned)(L & 7)) << ((L >> 3) - 3);
    unsigned y = 1u;
    while (rank_level(y) < L) ++y;  // y <= 8
    return y;
}

// The walk of a level-partitioned list may stop after a vector whose largest
// element x has rank_level(n - x) > L, L the level of the table's smallest key.
// rank_level(n - x) does not increase with x, so for 0 <= x < n that test is
// x < level_xthr(L, n): one compare per batch instead of a level computation.
__device__ __forceinline__ int level_xthr(int L, long long n) {
    const unsigned y = level_min_y(L + 1);
    if (y == 0u) return INT_MIN;
    const long long t = n - (long long)y + 1;
    return t < (long long)INT_MIN ? INT_MIN : (int)t;
}

// Binary-search mode (probe = 2, vertex-id lists): find x in the sorted
// segment; on a hit count it (per-vertex counter of x when PV) and return true.
template <bool PV>
__device__ __forceinline__ bool bsearch_hit(const Table& t, int x) {
    const int h = table_find_sorted(t.keys, t.len, x);
    if (h < 0) return false;
    if (PV) atomicAdd(&t.cnts[h], 1);
    return true;
}

// Lanes per partner for a list-length class c (lists of 2^c .. 2^(c+1)-1
// elements): one lane up to 2^(TC_CTA_LANE_SHIFT+1)-1 elements, then doubling
// up to a full warp, so that every lane of a task loads 2^(TC_CTA_LANE_SHIFT-2)
// to 2^(TC_CTA_LANE_SHIFT-1) aligned 16-byte vectors of its list (8 to 16 with
// the default shift of 5).  The shift is a compile-time constant: read from
// the kernel's arguments it costs 0.6 ms of k_count_cta on R-MAT s22.
__device__ __forceinline__ int class_lanes(int c) { return 1 << min(max(c - TC_CTA_LANE_SHIFT, 0), 5); }

// One warp intersects the partners pb+first, pb+first+stride, ... (in groups
// of 32, one partner per lane) with the table.
//
// The lists of the 32 partners are flattened into one sequence of
// tot = sum d+(q) elements; window k0 .. k0+31 puts element k0+lane on lane
// `lane`.  The owner of an element is found without a search: every partner
// marks the position where its list starts (all partner lists are non-empty,
// the partition guarantees it), the marks of a window are OR-reduced into a
// bit mask M, and the owner of position lane is (partners started before the
// window) + popc(M & lanes <= lane) - 1.  Each element is probed in the table;
// a ballot of the hits lets every partner lane count the hits that fall in
// its own range of the window, so per-partner counts need no atomics.
constexpr int kUnroll = 4;

template <bool PV, int PROBE>
__device__ __forceinline__ unsigned long long warp_partners(const CountArgs& a, const int* keys, int* cnts, int logS,
                                                            int len, int64_t pbase, int pb, int pe, int first,
                                                            int stride) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned le_mask = lane == 31 ? FULL : ((2u << lane) - 1u);
    unsigned long long acc = 0;
    for (int g0 = pb + first; g0 < pe; g0 += stride) {
        const int i = g0 + lane;
        const bool valid = i < pe;
        const int q = valid ? a.pcol[pbase + i] : 0;
        const int64_t qb = valid ? a.rpp[q] : 0;
        const int dq = valid ? (int)(a.rpp[q + 1] - qb) : 0;
        const int incl = warp_incl_scan_i(dq);
        const int tot = __shfl_sync(FULL, incl, 31);
        const int excl = incl - dq;
        const int64_t base = qb - excl;  // element k of partner q sits at colp[base + k]
        int myc = 0, P = 0;
        for (int k0 = 0; k0 < tot; k0 += 32 * kUnroll) {
            int w[kUnroll];
            bool in[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int s = excl - (k0 + 32 * u);
                const unsigned bit = (valid && s >= 0 && s < 32) ? (1u << s) : 0u;
                const unsigned M = __reduce_or_sync(FULL, bit);
                const int j = P + __popc(M & le_mask) - 1;
                P += __popc(M);
                const int64_t bj = __shfl_sync(FULL, base, j & 31);
                const int k = k0 + 32 * u + lane;
                in[u] = k < tot;
                w[u] = in[u] ? a.colp[bj + k] : 0;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                bool hit = false;
                if (in[u]) {
                    const int h = table_find_sorted(keys, len, w[u]);
                    if (h >= 0) {
                        hit = true;
                        if (PV) atomicAdd(&cnts[h], 1);
                    }
                }
                const unsigned hm = __ballot_sync(FULL, hit);
                if (hm) {
                    const int s = excl - (k0 + 32 * u);
                    const int lo = max(s, 0), hi = min(s + dq, 32);
                    if (lo < hi) {
                        const unsigned rm = (hi >= 32 ? FULL : ((1u << hi) - 1u)) & (FULL << lo);
                        myc += __popc(hm & rm);
                    }
                }
            }
        }
        if (valid && myc) {
            acc += (unsigned long long)myc;
            if (PV) atomicAdd(&a.t[q], (unsigned long long)myc);
        }
    }
    return acc;
}

// warp_partners over the padded rank-id lists, flattened by whole 16-byte
// vectors: window k0 .. k0+31 puts vector k0+lane of the 32 partners'
// concatenated vector sequence on lane `lane` (owner found as in
// warp_partners), and each lane probes the 4 elements of its vector in the
// zero-encoded hash table of the pivot (padding -1 never hits).  Per-partner
// hit counts come from one ballot per vector component.
#ifndef TC_WARP_VEC
#define TC_WARP_VEC 2
#endif
constexpr int kWarpVec = TC_WARP_VEC;

template <bool PV>
__device__ __forceinline__ unsigned long long warp_partners_vec(const CountArgs& a, const int* keys, int* cnts,
                                                                int logS, int64_t pbase, int pb, int pe) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned le_mask = lane == 31 ? FULL : ((2u << lane) - 1u);
    const int4* __restrict__ lv = reinterpret_cast<const int4*>(a.colr);
    unsigned long long acc = 0;
    // partner descriptors of the next group of 32 are loaded one group ahead
    int qn = 0, nvn = 0;
    int64_t qvn = 0;
    if (pb + lane < pe) {
        qn = a.pcol[pbase + pb + lane];
        const int2 d = a.pdesc[pbase + pb + lane];
        qvn = d.x;
        nvn = (d.y + 3) >> 2;
    }
    for (int g0 = pb; g0 < pe; g0 += 32) {
        const bool valid = g0 + lane < pe;
        const int q = qn;
        const int64_t qv = qvn;  // first vector of q's row
        const int nvq = nvn;     // >= 1: partner lists are non-empty
        if (g0 + 32 + lane < pe) {
            qn = a.pcol[pbase + g0 + 32 + lane];
            const int2 d = a.pdesc[pbase + g0 + 32 + lane];
            qvn = d.x;
            nvn = (d.y + 3) >> 2;
        } else {  // past the last partner: an empty descriptor
            qn = 0;
            qvn = 0;
            nvn = 0;
        }
        const int incl = warp_incl_scan_i(nvq);
        const int tot = __shfl_sync(FULL, incl, 31);
        const int excl = incl - nvq;
        const int64_t base = qv - excl;  // vector k of the flattened sequence owned by q is lv[base + k]
        int myc = 0, P = 0;
        for (int k0 = 0; k0 < tot; k0 += 32 * kWarpVec) {
            int4 w[kWarpVec];
#pragma unroll
            for (int u = 0; u < kWarpVec; ++u) {
                const int s = excl - (k0 + 32 * u);
                const unsigned bit = (valid && s >= 0 && s < 32) ? (1u << s) : 0u;
                const unsigned M = __reduce_or_sync(FULL, bit);
                const int j = P + __popc(M & le_mask) - 1;
                P += __popc(M);
                const int64_t bj = __shfl_sync(FULL, base, j & 31);
                const int k = k0 + 32 * u + lane;
                w[u] = (k < tot && dbg_ok((bj + k) * 4 + 3 < a.colr_len, TC_DEVERR_BOUNDS)) ? lv[bj + k]
                                                                                             : make_int4(-1, -1, -1, -1);
            }
#pragma unroll
            for (int u = 0; u < kWarpVec; ++u) {
                const int xs[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
                const int s = excl - (k0 + 32 * u);
                const int lo = max(s, 0), hi = min(s + nvq, 32);
                const unsigned rm = lo < hi ? ((hi >= 32 ? FULL : ((1u << hi) - 1u)) & (FULL << lo)) : 0u;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    bool hit = false;
                    if (xs[c] >= 0) {
                        const int h = table_find_z(keys, logS, xs[c]);
                        if (h >= 0) {
                            hit = true;
                            if (PV) atomicAdd(&cnts[h], 1);
                        }
                    }
                    const unsigned hm = __ballot_sync(FULL, hit);
                    myc += __popc(hm & rm);
                }
            }
        }
        if (valid && myc) {
            acc += (unsigned long long)myc;
            if (PV) atomicAdd(&a.t[q], (unsigned long long)myc);
        }
    }
    return acc;
}

// Binary-search mode: lane r of the G lanes that share one partner list
// (start qb, length dq in the unpadded vertex-id lists) probes the list's
// elements, reading it as aligned 16-byte vectors r, r+G, ... (the lists are
// padded by 4 elements at the end of the array), kVec vectors in flight, with
// a bounds test per element.  Returns this lane's hits.
template <bool PV>
__device__ __forceinline__ int probe_list_bsearch(const Table& tb, const int32_t* __restrict__ L, int64_t qb, int dq,
                                                  int r, int G) {
    const int s0 = (int)(qb & 3);
    const int4* __restrict__ lv = reinterpret_cast<const int4*>(L + (qb - s0));
    const int nv = (s0 + dq + 3) >> 2;
    int myc = 0;
    for (int v0 = r; v0 < nv; v0 += G * kVec) {
        int4 w[kVec];
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int vv = v0 + u * G;
            w[u] = (vv < nv && dbg_ok(qb - s0 + 4ll * vv + 3 < tb.llen, TC_DEVERR_BOUNDS)) ? lv[vv]
                                                                                           : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int j0 = 4 * (v0 + u * G) - s0;  // list position of w[u].x
            if ((unsigned)(j0 + 0) < (unsigned)dq && bsearch_hit<PV>(tb, w[u].x)) ++myc;
            if ((unsigned)(j0 + 1) < (unsigned)dq && bsearch_hit<PV>(tb, w[u].y)) ++myc;
            if ((unsigned)(j0 + 2) < (unsigned)dq && bsearch_hit<PV>(tb, w[u].z)) ++myc;
            if ((unsigned)(j0 + 3) < (unsigned)dq && bsearch_hit<PV>(tb, w[u].w)) ++myc;
        }
    }
    return myc;
}

// Shared-memory add under a predicate, with no branch around it: the per-hit
// counter update of a probe costs the same instructions whether it hits or not.
__device__ __forceinline__ void red_shared_if(bool p, const void* addr, unsigned v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(addr);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.shared.add.u32 [%0], %1;\n\t}" ::"r"(a), "r"(v),
        "r"((unsigned)p)
        : "memory");
}

// The probe of a 16-bit direct cell with per-vertex counts, as one predicated
// shared atomic: if off < span, add v to the 32-bit word at shared address
// addr and return its old value, else return 0.  The span test is the
// predicate itself, so a probe costs the offset, the address and the atomic.
__device__ __forceinline__ unsigned atom_probe(unsigned off, unsigned span, unsigned addr, unsigned v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\tmov.u32 %0, 0;\n\t@q atom.shared.add.u32 %0, [%3], %4;\n\t}"
        : "=r"(r)
        : "r"(off), "r"(span), "r"(addr), "r"(v)
        : "memory");
    return r;
}

// Probe one element x of a padded rank-id list (x = -1 is padding and never
// hits); returns 1 on a hit and counts it for x's per-vertex total when PV.
template <int MODE, bool PV>
__device__ __forceinline__ int probe1(const Table& t, int x) {
    if (MODE == kModeDirect32) {
        if (PV) {
            const unsigned off = min((unsigned)(x - t.lo), t.lim);
            if (!dbg_ok(off < (unsigned)t.ucap, TC_DEVERR_BOUNDS)) return 0;
            unsigned r;
            asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(r) : "r"(t.sbase + (off << 2)) : "memory");
            return (int)(r >> 31);
        }
        const unsigned off = (unsigned)(x - t.lo);
        const unsigned c = off < (unsigned)t.span ? t.cell32[off] : 0u;
        return c != 0u ? 1 : 0;
    } else if (MODE == kModeDirect) {
        const unsigned off = (unsigned)(x - t.lo);
        if (!dbg_ok(off >= (unsigned)t.span || (off >> 1) < (unsigned)t.ucap, TC_DEVERR_BOUNDS)) return 0;
        if (PV) {
            const unsigned sh = (off & 1u) << 4;
            return (int)((atom_probe(off, (unsigned)t.span, t.sbase + ((off << 1) & ~3u), 1u << sh) >> (15u + sh)) & 1u);
        }
        const unsigned c = off < (unsigned)t.span ? (unsigned)t.cell[off] : 0u;
        return c != 0u ? 1 : 0;
    } else if (MODE == kModeBitmap) {
        const unsigned off = (unsigned)(x - t.lo);
        const bool in = off < (unsigned)t.span && dbg_ok((off >> 5) < (unsigned)t.wmax, TC_DEVERR_BOUNDS);
        const unsigned word = in ? t.bits[off >> 5] : 0u;
        const unsigned b = off & 31u;
        const bool hit = (word >> b) & 1u;
        if (PV) {
            const int ord = hit ? (int)t.pre[off >> 5] + __popc(word & ((1u << b) - 1u)) : 0;
            red_shared_if(hit, t.cnts + ord, 1u);
        }
        return hit ? 1 : 0;
    } else {
        if (x < 0) return 0;
        const int h = table_find_z(t.keys, t.logS, x);
        if (h < 0 || !dbg_ok(h < t.ucap / 2, TC_DEVERR_BOUNDS)) return 0;
        if (PV) atomicAdd(&t.cnts[h], 1);
        return 1;
    }
}

// probe_list for the padded rank-id rows: the list starts 16-byte aligned and
// its last vector is filled up with -1, so every vector is probed whole.  The
// lane walks vectors nv-1-r, nv-1-r-G, ... (top down).  For a list partitioned
// by rank level, x_exit is the table's level_xthr and the walk stops after a
// batch whose lowest vector lies wholly in levels above that of the table's
// smallest key (everything further down is below the table); x_exit = INT_MIN
// walks the whole list.
template <int MODE, bool PV>
__device__ __forceinline__ int probe_list_padded(const Table& tb, const int32_t* __restrict__ L, int64_t qb, int dq,
                                                 int r, int G, int x_exit) {
    const int4* __restrict__ lv = reinterpret_cast<const int4*>(L + qb);
    const int nv = (dq + 3) >> 2;
    int myc = 0;
    for (int v0 = nv - 1 - r; v0 >= 0; v0 -= G * kVec) {
        int4 w[kVec];
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int vv = v0 - u * G;
            w[u] = (vv >= 0 && dbg_ok(qb + 4ll * vv + 3 < tb.llen, TC_DEVERR_BOUNDS)) ? lv[vv]
                                                                                      : make_int4(-1, -1, -1, -1);
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u)
            myc += probe1<MODE, PV>(tb, w[u].x) + probe1<MODE, PV>(tb, w[u].y) + probe1<MODE, PV>(tb, w[u].z) +
                   probe1<MODE, PV>(tb, w[u].w);
        const int4 t = w[kVec - 1];
        if (max(max(t.x, t.y), max(t.z, t.w)) < x_exit) break;
    }
    return myc;
}

// ---------------------------------------------------------------------------
// Staged partner lists (CTA-table kernel, lists of >= 4 lanes per partner)
//
// A warp task covers 32/G partners with G lanes each; the lanes of one partner
// walk its padded rank-id list top down in batches of 4 vectors per lane, so
// batch b of the task is, for every partner, the 4G vectors below the ones of
// batch b-1: at most 32 x 4 = 128 vectors (2 KB) in all.  Instead of loading them
// itself, the warp has lane 0 copy batch b+1 of every live partner from
// global into one of its two shared-memory slots with cp.async.bulk (one copy
// per partner, completing on the slot's mbarrier) before it probes batch b
// from the other slot, so the copy engine moves the lists while the lanes
// probe.  Each warp owns its two slots and two mbarriers and waits for its
// copies in the order it issued them, so a slot's phase parity always names
// the copy waited for.  A partner whose lowest vector of a batch lies wholly
// below the table is not copied again (everything further down is below it).
// ---------------------------------------------------------------------------
constexpr int kSlotVec = 128;                    // vectors (16 B) per staging slot
static_assert(32 * kVec <= kSlotVec, "a batch of a warp task fills at most one slot");
constexpr long long kWaitCycles = 2000000000ll;  // about one second at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// One thread's asynchronous copy of 4 or 8 bytes (aligned to their size)
// from global into shared memory; completes at cp.async.wait_all.
__device__ __forceinline__ void cp_async_g2s(void* sdst, const void* gsrc, int bytes) {
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned addr, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(addr),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned addr, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(unsigned dst, const void* src, unsigned bytes, unsigned mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

struct StageCtx {
    int4* buf;          // this warp's two slots (2 x kSlotVec vectors)
    unsigned bar;       // shared address of this warp's two mbarriers (8 bytes apart)
    unsigned issued;    // batches issued so far: batch k uses slot k & 1, phase parity (k >> 1) & 1
    bool failed;        // a wait gave up (TC_DEVERR_WAIT raised); the warp stops staging
};

// Lane 0 copies batch b of every live partner of the task into the next slot.
// All lanes take part (the partners' descriptors are broadcast from their
// first lanes); lane 0 alone issues the copies and the transaction count.
__device__ __forceinline__ void stage_issue(const int32_t* __restrict__ colr, StageCtx& st, int G, int ppt,
                                            int64_t qb, int nv, bool live, int b) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int W = kVec * G;
    const unsigned slot = st.issued & 1u;
    const unsigned bar = st.bar + 8u * slot;
    const unsigned dst0 = smem_u32(st.buf + (size_t)slot * kSlotVec);
    unsigned bytes = 0;
    __syncwarp();  // every lane is done with the batch this slot held before
    for (int sp = 0; sp < ppt; ++sp) {
        const int64_t q_b = __shfl_sync(FULL, qb, sp * G);
        const int q_nv = __shfl_sync(FULL, nv, sp * G);
        const int q_live = __shfl_sync(FULL, live ? 1 : 0, sp * G);
        const int hi = q_nv - b * W, lo = max(0, hi - W);
        if (lane == 0 && q_live && hi > 0) {
            const unsigned nb = (unsigned)(hi - lo) * 16u;
            bulk_copy_g2s(dst0 + (unsigned)(sp * W) * 16u, colr + q_b + 4ll * lo, nb, bar);
            bytes += nb;
        }
    }
    if (lane == 0) mbar_arrive_tx(bar, bytes);
    st.issued += 1;
}

// Every lane waits for batch k itself (so that each observes the copy's
// completion before reading the slot); bounded: past kWaitCycles the lane gives
// up, and the warp stops staging if any lane gave up (a warp-uniform decision).
__device__ __forceinline__ void stage_wait(StageCtx& st, unsigned k) {
    const unsigned bar = st.bar + 8u * (k & 1u), par = (k >> 1) & 1u;
    bool ok = mbar_test(bar, par);
    if (!ok) {
        const long long t0 = clock64();
        while (!(ok = mbar_test(bar, par)) && clock64() - t0 <= kWaitCycles) {
        }
    }
    if (__any_sync(0xffffffffu, !ok)) {
        if (!ok) raise_error(TC_DEVERR_WAIT);
        st.failed = true;
    }
}

// One warp task of G >= 4 lanes per partner, probed from the staged batches.
// Returns this lane's hits (summed over the partner's G lanes by the caller).
template <int MODE, bool PV>
__device__ __forceinline__ int probe_task_staged(const Table& tb, const int32_t* __restrict__ colr, StageCtx& st,
                                                 int G, int ppt, bool valid, int64_t qb, int dq, int x_exit) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, sub = lane / G, r = lane % G;
    const int W = kVec * G;
    const int nv = valid ? (dq + 3) >> 2 : 0;
    int nb = (nv + W - 1) / W;
    for (int o = 16; o; o >>= 1) nb = max(nb, __shfl_xor_sync(FULL, nb, o));
    bool live = nv > 0;
    int myc = 0;
    const unsigned gmask = (G >= 32 ? FULL : ((1u << G) - 1u)) << (sub * G);
    stage_issue(colr, st, G, ppt, qb, nv, live, 0);
    for (int b = 0; b < nb; ++b) {
        const unsigned k = st.issued - 1;  // this batch
        if (b + 1 < nb) stage_issue(colr, st, G, ppt, qb, nv, live, b + 1);
        stage_wait(st, k);
        if (st.failed) break;
        const int4* __restrict__ sv = st.buf + (size_t)(k & 1u) * kSlotVec + sub * W;
        const int hi = nv - b * W, lo = max(0, hi - W);
        bool stop = false;
        if (live && hi > 0) {
            int4 w[kVec];
#pragma unroll
            for (int u = 0; u < kVec; ++u) {
                const int vv = hi - 1 - r - u * G;
                w[u] = vv >= lo ? sv[vv - lo] : make_int4(-1, -1, -1, -1);
            }
#pragma unroll
            for (int u = 0; u < kVec; ++u)
                myc += probe1<MODE, PV>(tb, w[u].x) + probe1<MODE, PV>(tb, w[u].y) + probe1<MODE, PV>(tb, w[u].z) +
                       probe1<MODE, PV>(tb, w[u].w);
            const int4 t = w[kVec - 1];
            stop = max(max(t.x, t.y), max(t.z, t.w)) < x_exit || lo == 0;
        }
        // a partner stops once any of its lanes saw its lowest vector below the table
        // (or its list is used up); the next batch, already issued, is not probed
        const unsigned sm = __ballot_sync(FULL, stop);
        if (sm & gmask) live = false;
        if (!__any_sync(FULL, live)) {
            if (b + 1 < nb) stage_wait(st, k + 1);
            break;
        }
    }
    return myc;
}

// Intersect the item's partners [pb, pe) with the table.  Partners are taken
// pmax at a time, counting-sorted by length class, and cut into warp tasks of
// 32/G partners of one class with G lanes per partner (the dynamic grouping by
// list size of Sec. 4.2.2, inside one CTA).  Warps take tasks longest class
// first from a shared counter.  Every lane walks elements r, r+G, ... of its
// partner's list, so loads are contiguous per partner and hits of a partner
// stay in registers until a G-lane reduction.
template <bool PV, int MODE>
__device__ __forceinline__ unsigned long long cta_partners(const CountArgs& a, const int32_t* __restrict__ L,
                                                           const Table& tb, int64_t pbase, int pb, int pe, int pmax,
                                                           const CtaScratch& sc, StageCtx* st) {
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    unsigned long long acc = 0;
    constexpr int kPer = kCtaPer;  // partners per thread while sorting (pmax <= kPer * blockDim)
    for (int c0 = pb; c0 < pe; c0 += pmax) {
        const int NP = min(pmax, pe - c0);
        if (tid < kClasses) sc.ccnt[tid] = 0;
        if (tid == 0) sc.misc[0] = 0;
        __syncthreads();
        int rq[kPer], rd[kPer], rc[kPer], rs[kPer];
        int64_t rb[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * blockDim.x;
            rc[k] = -1;
            rq[k] = rd[k] = rs[k] = 0;
            rb[k] = 0;
            if (i < NP) {
                rq[k] = a.pcol[pbase + c0 + i];
                if (MODE == kModeBsearch) {
                    rb[k] = a.rpp[rq[k]];
                    rd[k] = a.dp[rq[k]];
                } else {  // the descriptor the build stored beside the partner
                    const int2 d = a.pdesc[pbase + c0 + i];
                    rb[k] = (int64_t)d.x << 2;
                    rd[k] = d.y;
                }
                rc[k] = min(kClasses - 1, 31 - __clz(rd[k]));
                rs[k] = atomicAdd(&sc.ccnt[rc[k]], 1);
            }
        }
        __syncthreads();
        if (tid == 0) {
            int pos = 0, task = 0;
            for (int c = kClasses - 1; c >= 0; --c) {
                sc.coff[c] = pos;
                sc.toff[c] = task;
                const int ppt = 32 / class_lanes(c);
                pos += sc.ccnt[c];
                task += (sc.ccnt[c] + ppt - 1) / ppt;
            }
            sc.misc[1] = task;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (rc[k] >= 0) {
                const int pos = sc.coff[rc[k]] + rs[k];
                sc.q[pos] = rq[k];
                sc.qb[pos] = rb[k];
                sc.dq[pos] = rd[k];
            }
        }
        const int NT = sc.misc[1];
        for (int t = tid; t < NT; t += blockDim.x) {
            int c = kClasses - 1;
            while (c > 0 && sc.toff[c - 1] <= t) --c;  // task ranges grow as the class falls
            sc.tcls[t] = (unsigned char)c;
        }
        __syncthreads();
        for (;;) {
            int t = 0;
            if (lane == 0) t = atomicAdd(&sc.misc[0], 1);
            t = __shfl_sync(FULL, t, 0);
            if (t >= NT) break;
            const int c = sc.tcls[t];
            const int G = class_lanes(c);
            const int ppt = 32 / G;
            const int sub = lane / G, r = lane % G;
            const int i = sc.coff[c] + (t - sc.toff[c]) * ppt + sub;
            const bool valid = i < sc.coff[c] + sc.ccnt[c];
            const int dq = valid ? sc.dq[i] : 0;
            const int64_t qb = valid ? sc.qb[i] : 0;
            // level-partitioned lists (kSortedMin <= d+ <= kSortedMax) may stop below the table
            const int x_exit = (dq >= kSortedMin && dq <= kSortedMax) ? tb.xthr : INT_MIN;
            int myc;
            if constexpr (MODE == kModeBsearch) myc = probe_list_bsearch<PV>(tb, L, qb, dq, r, G);
            else if (st && G >= 4 && !st->failed) myc = probe_task_staged<MODE, PV>(tb, L, *st, G, ppt, valid, qb, dq, x_exit);
            else myc = probe_list_padded<MODE, PV>(tb, L, qb, dq, r, G, x_exit);
            for (int off = G >> 1; off; off >>= 1) myc += __shfl_xor_sync(FULL, myc, off);
            if (r == 0 && valid && myc) {
                acc += (unsigned long long)myc;
                if (PV) atomicAdd(&a.t[sc.q[i]], (unsigned long long)myc);
            }
        }
        __syncthreads();
    }
    return acc;
}

// ints of the table region: hash (keys + counts, 8*cap) or bitmap (words,
// 16-bit word prefixes, counts), whichever is larger
static int cta_table_ints(int cap, int bitmap_bits) {
    const int words = bitmap_bits / 32;
    const int bm = words + (words + 1) / 2 + cap;
    return (std::max(8 * cap, bm) + 3) & ~3;  // whole 16-byte vectors (span clears)
}

// partners sorted per sub-chunk: kCtaPer per thread
__host__ __device__ __forceinline__ size_t cta_smem_bytes_dev(int u_ints, int threads) {
    const int pmax = kCtaPer * threads;
    return (size_t)((u_ints + 1) & ~1) * sizeof(int) + (size_t)pmax * (sizeof(int64_t) + 2 * sizeof(int) + 1) +
           (3 * kClasses + 4 + 33) * sizeof(int) + 16;
}
static size_t cta_smem_bytes(int u_ints, int threads) {
    const int pmax = kCtaPer * threads;
    return (size_t)((u_ints + 1) & ~1) * sizeof(int) + (size_t)pmax * (sizeof(int64_t) + 2 * sizeof(int) + 1) +
           (3 * kClasses + 4 + 33) * sizeof(int) + 16;
}

// staged kernel: two slots and two mbarriers per warp after the partner scratch
static size_t cta_stage_offset(int u_ints, int threads) { return (cta_smem_bytes(u_ints, threads) + 127) & ~(size_t)127; }
static size_t cta_stage_bytes(int u_ints, int threads) {
    return cta_stage_offset(u_ints, threads) + (size_t)(threads / 32) * (2 * kSlotVec * 16 + 16);
}

__device__ __forceinline__ void block_minmax(int& mn, int& mx, int* red) {
    for (int o = 16; o; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[w] = mn; red[32 + w] = mx; }
    __syncthreads();
    mn = 0x7fffffff;
    mx = -1;
    for (int i = 0; i < nw; ++i) { mn = min(mn, red[i]); mx = max(mx, red[32 + i]); }
    __syncthreads();
}

// BIG = false: at most 256 threads, registers capped for 4 resident CTAs per SM
// (3 with STAGED partner lists, whose slots take 32 KB more shared memory)
template <bool PV, int PROBE, bool BIG, bool STAGED>
#ifndef TC_CTA_MIN_BLOCKS
#define TC_CTA_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(BIG ? 1024 : 256, BIG ? 1 : (STAGED ? 3 : TC_CTA_MIN_BLOCKS)) k_count_cta(CountArgs a) {
    extern __shared__ __align__(16) int smem[];
    int* U = smem;
    CtaScratch sc;
    const int pmax = kCtaPer * blockDim.x;
    sc.qb = reinterpret_cast<int64_t*>(smem + ((a.u_ints + 1) & ~1));
    sc.q = reinterpret_cast<int*>(sc.qb + pmax);
    sc.dq = sc.q + pmax;
    sc.ccnt = sc.dq + pmax;
    sc.coff = sc.ccnt + kClasses;
    sc.toff = sc.coff + kClasses;
    sc.misc = sc.toff + kClasses;
    sc.scan = sc.misc + 4;
    sc.tcls = reinterpret_cast<unsigned char*>(sc.scan + 33);
    // staged partner lists: this warp's two slots and mbarriers
    StageCtx stage{};
    StageCtx* st = nullptr;
    if (STAGED) {
        const size_t off = (cta_smem_bytes_dev(a.u_ints, blockDim.x) + 127) & ~(size_t)127;
        char* base = reinterpret_cast<char*>(smem) + off;
        const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        stage.buf = reinterpret_cast<int4*>(base) + (size_t)warp * 2 * kSlotVec;
        unsigned long long* bars = reinterpret_cast<unsigned long long*>(base + (size_t)nw * 2 * kSlotVec * 16);
        stage.bar = smem_u32(bars + 2 * warp);
        stage.issued = 0;
        stage.failed = false;
        if ((threadIdx.x & 31) == 0) {
            mbar_init(stage.bar, 1);
            mbar_init(stage.bar + 8u, 1);
            // the initialised barriers are visible to the copy engine (async proxy)
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncwarp();
        st = &stage;
    }
    __shared__ int s_red[64];
    __shared__ unsigned long long s_acc;
    // the next work item, fetched one iteration ahead by thread 0 so that the
    // queue atomic and the dependent descriptor loads overlap the current item
    __shared__ Item s_cur;
    __shared__ long long s_r0, s_r1, s_prp;
    __shared__ int2 s_span;
    __shared__ int s_valid;
#if TC_CTA_ITEM_PREFETCH
    // the next item's row offset, d+, partner offset and rank span, copied
    // into shared memory by thread 0 with cp.async while the current item's
    // partners are walked (no registers held, no stall until the item ends)
    __shared__ long long s_nrpp, s_nprp;
    __shared__ int2 s_nspan;
    __shared__ int s_ndp;
#endif
    const int lane = threadIdx.x & 31;
    // hash mode probes rank ids (so that a short span can use the bitmap);
    // the binary-search mode probes the id-sorted lists
    const int32_t* __restrict__ L = PROBE == kProbeHash ? a.colr : a.colp;
    constexpr bool kPadded = PROBE == kProbeHash;  // colr rows (colr_row) or colp rows (rpp)
    const unsigned long long n_all = min(*a.n_items, a.items_cap);
    const unsigned long long it_lo = n_all * a.shard / a.nshards;
    const unsigned long long n_items = n_all * (a.shard + 1) / a.nshards;
    const int wmax = a.bitmap_bits / 32;
    for (int i = threadIdx.x; i < a.u_ints; i += blockDim.x) U[i] = 0;
    if (threadIdx.x == 0) {
        const unsigned long long it = it_lo + atomicAdd(a.queue, 1u);
        s_valid = it < n_items;
        if (s_valid) {
            s_cur = a.items[it];
            s_r0 = kPadded ? colr_row(a.rpp, s_cur.p) : a.rpp[s_cur.p];
            s_r1 = s_r0 + a.dp[s_cur.p];
            s_prp = a.prp[s_cur.p];
            s_span = a.rspan[s_cur.p];
        }
    }
    for (;;) {
        __syncthreads();
        if (!s_valid) break;
        const Item item = s_cur;
        const int p = item.p;
        const int64_t r0 = s_r0, r1 = s_r1, pbase = s_prp;
        const int2 pspan = s_span;
        __syncthreads();  // everyone has read the current item
        unsigned long long nit = 0;
        Item nitem{};
        if (threadIdx.x == 0) {
            s_acc = 0;
            nit = it_lo + atomicAdd(a.queue, 1u);
            if (nit < n_items) nitem = a.items[nit];
        }
        const int64_t lb = r0 + (int64_t)item.seg * a.cap;
        const int len = (int)min((int64_t)a.cap, r1 - lb);
        Table tb{};
        tb.len = len;
        tb.xthr = INT_MIN;
        tb.sbase = (unsigned)__cvta_generic_to_shared(U);
        tb.ucap = a.u_ints;
        tb.wmax = wmax;
        tb.llen = PROBE == kProbeHash ? a.colr_len : a.colp_len;
        if (TC_DEBUG) {  // the table region is all zeros at the start of every item
            bool dirty = false;
            for (int i = threadIdx.x; i < a.u_ints; i += blockDim.x) dirty |= U[i] != 0;
            if (dirty) raise_error(TC_DEVERR_DIRTY);
        }
        int mode = PROBE == kProbeHash ? kModeHash : kModeBsearch;
        if (PROBE == kProbeHash && a.bitmap_bits > 0) {
            int mn, mx;
            if (r1 - r0 == len) {  // the whole row: its span is known
                mn = pspan.x;
                mx = pspan.y;
            } else {
                mn = 0x7fffffff;
                mx = -1;
                for (int i = threadIdx.x; i < len; i += blockDim.x) {
                    const int x = L[lb + i];
                    mn = min(mn, x);
                    mx = max(mx, x);
                }
                block_minmax(mn, mx, s_red);
            }
            if (mx - mn < a.direct_span / 2 && mx - mn + 1 + 32 <= a.u_ints) {  // + the dummy cells
                mode = kModeDirect32;
                tb.lo = mn;
                tb.span = mx - mn + 1;
            } else if (mx - mn < a.direct_span && (mx - mn + 2) / 2 <= a.u_ints && item.pe - item.pb < 0x8000) {
                mode = kModeDirect;
                tb.lo = mn;
                tb.span = mx - mn + 1;
            } else if (mx - mn < a.bitmap_bits) {
                mode = kModeBitmap;
                tb.lo = mn;
                tb.span = mx - mn + 1;
            }
            if (mx >= 0) tb.xthr = level_xthr(rank_level((unsigned)(a.n - mn)), a.n);
            tb.lim = (unsigned)tb.span + (unsigned)lane;
        }
        // the table region is all zeros here: every item resets what it set
        int nflush = 0;
        if (mode == kModeDirect32) {
            tb.cell32 = reinterpret_cast<unsigned*>(U);
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const unsigned off = (unsigned)(L[lb + i] - tb.lo);
                if (dbg_ok(off < (unsigned)tb.span, TC_DEVERR_BOUNDS)) tb.cell32[off] = kMark32;
            }
        } else if (mode == kModeDirect) {
            tb.cell = reinterpret_cast<unsigned short*>(U);
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const unsigned off = (unsigned)(L[lb + i] - tb.lo);
                if (dbg_ok(off < (unsigned)tb.span, TC_DEVERR_BOUNDS)) tb.cell[off] = (unsigned short)kMark16;
            }
        } else if (mode == kModeBitmap) {
            const int W = (tb.span + 31) >> 5;
            unsigned* bits = reinterpret_cast<unsigned*>(U);
            unsigned short* pre = reinterpret_cast<unsigned short*>(U + wmax);
            tb.bits = bits;
            tb.pre = pre;
            tb.cnts = U + wmax + (wmax + 1) / 2;
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const unsigned off = (unsigned)(L[lb + i] - tb.lo);
                atomicOr(&bits[off >> 5], 1u << (off & 31u));
            }
            __syncthreads();
            if (PV) {  // prefix of set bits per word
                const int per = (W + blockDim.x - 1) / blockDim.x;
                const int w0 = threadIdx.x * per, w1 = min(W, w0 + per);
                int c = 0;
                for (int i = w0; i < w1; ++i) c += __popc(bits[i]);
                int tot;
                int run = block_excl_scan_i(c, sc.scan, &tot);
                for (int i = w0; i < w1; ++i) {
                    pre[i] = (unsigned short)run;
                    run += __popc(bits[i]);
                }
            }
        } else if (mode == kModeHash) {
            int* keys = U;
            tb.keys = keys;
            tb.cnts = U + 4 * a.cap;
            tb.logS = max(5, 32 - __clz(4 * len - 1));  // load factor <= 1/4
            for (int i = threadIdx.x; i < len; i += blockDim.x) table_insert_z(keys, tb.logS, L[lb + i]);
            nflush = 1 << tb.logS;
        } else {
            int* keys = U;
            tb.keys = keys;
            tb.cnts = U + 4 * a.cap;
            tb.logS = 0;
            for (int i = threadIdx.x; i < len; i += blockDim.x) keys[i] = L[lb + i];
            nflush = len;
        }
        __syncthreads();
        unsigned long long acc;
#if TC_CTA_ITEM_PREFETCH
        if (threadIdx.x == 0 && nit < n_items) {
            cp_async_g2s(&s_nrpp, a.rpp + nitem.p, 8);
            cp_async_g2s(&s_ndp, a.dp + nitem.p, 4);
            cp_async_g2s(&s_nprp, a.prp + nitem.p, 8);
            cp_async_g2s(&s_nspan, a.rspan + nitem.p, 8);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
#endif
        if (mode == kModeDirect32) acc = cta_partners<PV, kModeDirect32>(a, L, tb, pbase, item.pb, item.pe, pmax, sc, st);
        else if (mode == kModeDirect) acc = cta_partners<PV, kModeDirect>(a, L, tb, pbase, item.pb, item.pe, pmax, sc, st);
        else if (mode == kModeBitmap) acc = cta_partners<PV, kModeBitmap>(a, L, tb, pbase, item.pb, item.pe, pmax, sc, st);
        else if (mode == kModeHash) acc = cta_partners<PV, kModeHash>(a, L, tb, pbase, item.pb, item.pe, pmax, sc, st);
        else acc = cta_partners<PV, kModeBsearch>(a, L, tb, pbase, item.pb, item.pe, pmax, sc, st);
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) atomicAdd(&s_acc, acc);
        __syncthreads();
        // per-vertex counts of the table's keys, and reset of what this item set
        if (mode == kModeDirect32 || mode == kModeDirect) {
            if (PV) {
                for (int i = threadIdx.x; i < len; i += blockDim.x) {
                    const int x = L[lb + i];
                    const unsigned c = mode == kModeDirect32 ? tb.cell32[x - tb.lo] & ~kMark32
                                                             : (unsigned)tb.cell[x - tb.lo] & ~kMark16;
                    if (c) atomicAdd(&a.t_rank[x], (unsigned long long)c);
                }
                __syncthreads();
                // clear the whole span (junk counts of non-keys included)
                const int nz = mode == kModeDirect32 ? (tb.span + 32 + 3) >> 2 : (tb.span + 7) >> 3;
                uint4* z = reinterpret_cast<uint4*>(U);
                for (int i = threadIdx.x; i < nz; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
            } else if (mode == kModeDirect32) {
                for (int i = threadIdx.x; i < len; i += blockDim.x) tb.cell32[L[lb + i] - tb.lo] = 0u;
            } else {
                for (int i = threadIdx.x; i < len; i += blockDim.x) tb.cell[L[lb + i] - tb.lo] = 0;
            }
        } else if (mode == kModeBitmap) {
            if (PV) {
                for (int i = threadIdx.x; i < len; i += blockDim.x) {
                    const int x = L[lb + i];
                    const unsigned off = (unsigned)(x - tb.lo);
                    const unsigned word = tb.bits[off >> 5];
                    const int ord = (int)tb.pre[off >> 5] + __popc(word & ((1u << (off & 31u)) - 1u));
                    const int c = tb.cnts[ord];
                    if (c) atomicAdd(&a.t_rank[x], (unsigned long long)c);
                }
                __syncthreads();
                for (int i = threadIdx.x; i < len; i += blockDim.x) tb.cnts[i] = 0;
                unsigned short* pre = const_cast<unsigned short*>(tb.pre);
                for (int i = threadIdx.x; i < ((tb.span + 31) >> 5); i += blockDim.x) pre[i] = 0;
            }
            for (int i = threadIdx.x; i < len; i += blockDim.x)
                const_cast<unsigned*>(tb.bits)[(unsigned)(L[lb + i] - tb.lo) >> 5] = 0u;
        } else {
            for (int i = threadIdx.x; i < nflush; i += blockDim.x) {
                if (PV) {
                    const int c = tb.cnts[i];
                    if (c) {
                        const int x = mode == kModeHash ? tb.keys[i] - 1 : tb.keys[i];
                        if (PROBE == kProbeHash) atomicAdd(&a.t_rank[x], (unsigned long long)c);
                        else atomicAdd(&a.t[x], (unsigned long long)c);
                        tb.cnts[i] = 0;
                    }
                }
                if (mode == kModeHash) const_cast<int*>(tb.keys)[i] = 0;
            }
        }
        if (threadIdx.x == 0) {
            if (s_acc) {
                const int g = a.row_graph ? a.row_graph[p] : 0;
                atomicAdd(&a.totals[g], s_acc);
                if (PV) atomicAdd(&a.t[p], s_acc);
            }
            s_valid = nit < n_items;
            if (s_valid) {
                s_cur = nitem;
#if TC_CTA_ITEM_PREFETCH
                asm volatile("cp.async.wait_all;" ::: "memory");
                const int64_t rp_n = s_nrpp;
                s_r0 = kPadded ? colr_row_of(rp_n, nitem.p) : rp_n;
                s_r1 = s_r0 + s_ndp;
                s_prp = s_nprp;
                s_span = s_nspan;
#else
                s_r0 = kPadded ? colr_row(a.rpp, nitem.p) : a.rpp[nitem.p];
                s_r1 = s_r0 + a.dp[nitem.p];
                s_prp = a.prp[nitem.p];
                s_span = a.rspan[nitem.p];
#endif
            }
        }
    }
}

// ---------------------------------------------------------------------------
// warp-table kernel: each warp owns a table of 2*wcap slots
// ---------------------------------------------------------------------------
#ifndef TC_WARP_MIN_BLOCKS
#define TC_WARP_MIN_BLOCKS 4
#endif
template <bool PV, int PROBE>
__global__ void __launch_bounds__(256, TC_WARP_MIN_BLOCKS) k_count_warp(CountArgs a, int wcap) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_warp = 8 * wcap;
    int* keys = smem + warp * per_warp;
    int* cnts = keys + 4 * wcap;
    const unsigned long long n_all = min(*a.n_items, a.items_cap);
    const unsigned long long it_lo = n_all * a.shard / a.nshards;
    const unsigned long long n_items = n_all * (a.shard + 1) / a.nshards;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = it_lo + atomicAdd(a.queue, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const Item item = a.items[it];
        const int p = item.p;
        if (PROBE == kProbeHash) {
            // rank-id hash of N+(p) (keys x+1, 0 = empty); partners' padded rank-id lists
            const int64_t lb = colr_row(a.rpp, p);
            const int len = a.dp[p];
            const int logS = max(5, 32 - __clz(4 * len - 1));  // load factor <= 1/4
            const int S = 1 << logS;
            for (int i = lane; i < S; i += 32) {
                keys[i] = 0;
                if (PV) cnts[i] = 0;
            }
            __syncwarp();
            for (int i = lane; i < len; i += 32) table_insert_z(keys, logS, a.colr[lb + i]);
            __syncwarp();
            unsigned long long acc = warp_partners_vec<PV>(a, keys, cnts, logS, a.prp[p], item.pb, item.pe);
            __syncwarp();
            if (PV) {
                for (int i = lane; i < S; i += 32) {
                    const int c = cnts[i];
                    if (c) atomicAdd(&a.t_rank[keys[i] - 1], (unsigned long long)c);
                }
            }
            acc = warp_sum_u64(acc);
            if (lane == 0 && acc) {
                const int g = a.row_graph ? a.row_graph[p] : 0;
                atomicAdd(&a.totals[g], acc);
                if (PV) atomicAdd(&a.t[p], acc);
            }
            __syncwarp();
            continue;
        }
        const int64_t lb = a.rpp[p];
        const int len = (int)(a.rpp[p + 1] - lb);
        int logS, S;
        {
            logS = 0;
            S = len;
            for (int i = lane; i < len; i += 32) {
                keys[i] = a.colp[lb + i];
                if (PV) cnts[i] = 0;
            }
        }
        __syncwarp();
        unsigned long long acc =
            warp_partners<PV, PROBE>(a, keys, cnts, logS, len, a.prp[p], item.pb, item.pe, 0, 32);
        __syncwarp();
        if (PV) {
            for (int i = lane; i < S; i += 32) {
                const int c = cnts[i];
                if (c) atomicAdd(&a.t[keys[i]], (unsigned long long)c);
            }
        }
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) {
            const int g = a.row_graph ? a.row_graph[p] : 0;
            atomicAdd(&a.totals[g], acc);
            if (PV) atomicAdd(&a.t[p], acc);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// TwoSmall: a group of L = small_lanes threads per source row (L = 1: one
// thread per row), lane j of the group merging the row's edges j, j+L, ...:
// a sorted merge of two short vertex-id rows per edge.  The kernel needs few
// registers, so many resident threads hide the latency of the merge's loads.
// STEP (chosen per launch, small_max > 8): a branch-free merge step that
// carries both current elements and reloads only the side that moved.  On
// lists of up to 32 entries (BA graphs) it takes count_small from 17.4 to
// 14.8 ms; on lists of at most 8 the plain loop is as fast (R-MAT s22) or
// faster (a grid's 1-5 entries: 0.47 against 0.57 ms).
// ---------------------------------------------------------------------------
template <bool PV, bool STEP>
__global__ void __launch_bounds__(256) k_count_small(CountArgs a) {
    __shared__ unsigned long long s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    unsigned long long acc = 0;
    const int sm = a.small_max;
    const int lg = 31 - __clz(a.small_lanes);
    const int sub = (int)(threadIdx.x & (unsigned)(a.small_lanes - 1));
    const int64_t u_lo = a.n * a.shard / a.nshards, u_hi = a.n * (a.shard + 1) / a.nshards;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> lg;
    for (int64_t u = u_lo + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> lg); u < u_hi; u += stride) {
        const int du = a.dp[u];
        if (du < 2 || du > sm) continue;
        const int64_t ub = a.rpp[u];
        unsigned long long cu = 0;
        for (int i = sub; i < du; i += a.small_lanes) {
            const int v = a.colp[ub + i];
            if (!dbg_ok(v >= 0 && v < a.n, TC_DEVERR_BOUNDS)) continue;
            const int dv = a.dp[v];
            if (dv == 0 || dv > sm) continue;
            const int64_t vb = a.rpp[v];
            if (!dbg_ok(ub + du <= a.colp_len && vb + dv <= a.colp_len, TC_DEVERR_BOUNDS)) continue;
            int x = 0, y = 0, c = 0;
            if (STEP) {  // both lists are non-empty here: d+(u) >= 2, d+(v) >= 1
                int xa = a.colp[ub], yb = a.colp[vb];
                while (x < du && y < dv) {
                    const bool eq = xa == yb, ax = xa <= yb, ay = yb <= xa;
                    if (PV && eq) atomicAdd(&a.t[xa], 1ull);
                    c += eq;
                    x += ax;
                    y += ay;
                    if (ax && x < du) xa = a.colp[ub + x];
                    if (ay && y < dv) yb = a.colp[vb + y];
                }
            } else {
                while (x < du && y < dv) {
                    const int xa = a.colp[ub + x], yb = a.colp[vb + y];
                    if (xa < yb) ++x;
                    else if (xa > yb) ++y;
                    else {
                        ++c;
                        if (PV) atomicAdd(&a.t[xa], 1ull);
                        ++x;
                        ++y;
                    }
                }
            }
            if (c) {
                cu += (unsigned long long)c;
                if (PV) atomicAdd(&a.t[v], (unsigned long long)c);
            }
        }
        if (cu) {  // this lane's share of u's count
            if (PV) atomicAdd(&a.t[u], cu);
            if (a.row_graph) atomicAdd(&a.totals[a.row_graph[u]], cu);
            else acc += cu;
        }
    }
    if (!a.row_graph) {
        acc = warp_sum_u64(acc);
        if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&s_acc, acc);
        __syncthreads();
        if (threadIdx.x == 0 && s_acc) atomicAdd(&a.totals[0], s_acc);
    }
}

// ---------------------------------------------------------------------------
// Merge-path class: one warp per oriented edge (u, v) with balanced lists
// (the paper's TwoLarge intersection, Sec. 4.2.2, with the merge path split
// evenly over the 32 lanes).  Both lists are N+ rows of the oriented CSR in
// ascending vertex id.  Lane l takes diagonals [l L/32, (l+1) L/32) of the
// merge path of length L = |N+(u)| + |N+(v)|, finds its start by binary search
// (A = N+(u) is taken first on ties, so a common w is counted when its copy in
// A is consumed, by exactly one lane) and walks its diagonals.
// ---------------------------------------------------------------------------
template <bool PV>
__global__ void __launch_bounds__(256) k_count_merge(CountArgs a, const int2* __restrict__ medge,
                                                     const unsigned long long* __restrict__ n_medge,
                                                     unsigned long long cap) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned long long n_all = min(*n_medge, cap);
    const unsigned long long e_lo = n_all * a.shard / a.nshards, e_hi = n_all * (a.shard + 1) / a.nshards;
    const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (unsigned long long e = e_lo + warp; e < e_hi; e += nwarps) {
        const int2 uv = medge[e];
        if (!dbg_ok(uv.x >= 0 && uv.x < a.n && uv.y >= 0 && uv.y < a.n, TC_DEVERR_BOUNDS)) continue;
        const int64_t ab = a.rpp[uv.x], bb = a.rpp[uv.y];
        const int na = (int)(a.rpp[uv.x + 1] - ab), nb = (int)(a.rpp[uv.y + 1] - bb);
        if (!dbg_ok(ab + na <= a.colp_len && bb + nb <= a.colp_len, TC_DEVERR_BOUNDS)) continue;
        const int32_t* __restrict__ A = a.colp + ab;
        const int32_t* __restrict__ Bv = a.colp + bb;
        const int L = na + nb;
        const int d0 = (int)(((long long)L * lane) >> 5), d1 = (int)(((long long)L * (lane + 1)) >> 5);
        // i = number of A elements among the first d0 merged ones
        int lo = max(0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= Bv[d0 - mid - 1]) lo = mid + 1;
            else hi = mid;
        }
        int i = lo, j = d0 - lo, c = 0;
        for (int step = d0; step < d1; ++step) {
            const int x = i < na ? A[i] : INT_MAX;
            const int y = j < nb ? Bv[j] : INT_MAX;
            if (x <= y) {
                if (x == y) {
                    ++c;
                    if (PV) atomicAdd(&a.t[x], 1ull);
                }
                ++i;
            } else {
                ++j;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        if (lane == 0 && c) {
            if (PV) {
                atomicAdd(&a.t[uv.x], (unsigned long long)c);
                atomicAdd(&a.t[uv.y], (unsigned long long)c);
            }
            if (a.row_graph) atomicAdd(&a.totals[a.row_graph[uv.x]], (unsigned long long)c);
            else acc += (unsigned long long)c;
        }
    }
    if (!a.row_graph && lane == 0 && acc) atomicAdd(&a.totals[0], acc);
}

// The table keys' counts were accumulated by rank id (a pivot segment's keys
// are rank ids of a short span, so those atomics share cache lines and need no
// rank -> vertex lookup); t[perm[r]] += t_rank[r] folds them into t.
__global__ void k_fold_rank_counts(int64_t n, const int32_t* __restrict__ perm,
                                   const unsigned long long* __restrict__ t_rank, unsigned long long* __restrict__ t) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = t_rank[r];
        if (c) t[perm[r]] += c;  // perm is a bijection: one writer per vertex
    }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------
static int pow2ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <bool PV, int PROBE>
static cudaError_t launch_tables(tc_ctx* ctx, const CountArgs& base, const tc_ocsr* o, unsigned* queues, int num_sms,
                                 const Tuning& tun, cudaStream_t s) {
    // warp-table items
    {
        PhaseScope ph(ctx, kPhCountWarp, s);
        TC_LAUNCH(ctx);
        CountArgs a = base;
        a.items = o->items_warp;
        a.n_items = &o->dc->n_items_warp;
        a.items_cap = (unsigned long long)o->items_warp_cap;
        a.queue = queues + 0;
        const int wcap = std::max(16, pow2ceil(tun.warp_max));
        // 32*wcap bytes of table per warp; up to 8 warps per CTA within 192 KB
        const int wpb = std::max(1, std::min(8, (192 * 1024) / (32 * wcap)));
        const size_t smem = (size_t)wpb * (8 * wcap) * sizeof(int);
        auto kern = k_count_warp<PV, PROBE>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpb, smem);
        kern<<<(unsigned)(num_sms * std::max(per_sm, 1)), 32 * wpb, smem, s>>>(a, wcap);
    }
    // CTA-table items
    {
        PhaseScope ph(ctx, kPhCountCta, s);
        TC_LAUNCH(ctx);
        CountArgs a = base;
        a.items = o->items_cta;
        a.n_items = &o->dc->n_items_cta;
        a.items_cap = (unsigned long long)o->items_cta_cap;
        a.queue = queues + 1;
        a.u_ints = cta_table_ints(a.cap, a.bitmap_bits);
        const bool staged = PROBE == kProbeHash && tun.stage > 0 && tun.cta_threads <= 256;
        const size_t smem = staged ? cta_stage_bytes(a.u_ints, tun.cta_threads) : cta_smem_bytes(a.u_ints, tun.cta_threads);
        auto kern = staged ? k_count_cta<PV, PROBE, false, true>
                           : (tun.cta_threads <= 256 ? k_count_cta<PV, PROBE, false, false> : k_count_cta<PV, PROBE, true, false>);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tun.cta_threads, smem);
        kern<<<(unsigned)(num_sms * std::max(per_sm, 1)), tun.cta_threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

tc_status count_device(tc_ctx* ctx, const tc_ocsr* o, unsigned long long* totals, unsigned long long* per_vertex,
                       cudaStream_t s, int shard, int nshards) {
    const Tuning& tun = o->tun;
    const int64_t G = o->G > 0 ? o->G : 1;
    unsigned* queues = nullptr;
    unsigned long long* t_rank = nullptr;
    {
        PhaseScope ph(ctx, kPhCountInit, s);
        cudaError_t e = cudaMemsetAsync(totals, 0, sizeof(unsigned long long) * G, s);
        if (e == cudaSuccess && per_vertex && o->n > 0)
            e = cudaMemsetAsync(per_vertex, 0, sizeof(unsigned long long) * o->n, s);
        if (e != cudaSuccess) return cuda_err(ctx, e, "count: memset");
        if (o->n == 0 || o->m == 0) return TC_OK;
        e = dev_alloc((void**)&queues, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return set_err(ctx, TC_ERR_OOM, "count: queue allocation failed");
        cudaMemsetAsync(queues, 0, 2 * sizeof(unsigned), s);
        if (per_vertex) {
            e = dev_alloc((void**)&t_rank, sizeof(unsigned long long) * (size_t)o->n, s);
            if (e != cudaSuccess) {
                dev_free(queues, s);
                return set_err(ctx, TC_ERR_OOM, "count: rank-count allocation failed");
            }
            cudaMemsetAsync(t_rank, 0, sizeof(unsigned long long) * (size_t)o->n, s);
        }
    }
    cudaError_t e = cudaSuccess;

    CountArgs a{};
    a.rpp = o->rpp;
    a.colp = o->colp;
    a.dp = o->dplus;
    a.prp = o->prp;
    a.pcol = o->pcol;
    a.pdesc = o->pdesc;
    a.totals = totals;
    a.t = per_vertex;
    a.t_rank = t_rank;
    a.row_graph = o->row_graph;
    a.n = o->n;
    a.cap = tun.table_cap;
    a.small_max = tun.small_max;
    a.small_lanes = tun.small_lanes;
    a.shard = shard;
    a.nshards = nshards;
    a.colr = o->colr;
    a.colr_len = std::max<int64_t>(o->m, 1) + 3 * o->n + 4;
    a.colp_len = std::max<int64_t>(o->m, 1) + 4;
    a.perm = o->perm;
    a.rspan = o->rspan;
    a.bitmap_bits = tun.bitmap_bits;
    a.direct_span = tun.direct_span;
    const int ns = ctx->num_sms;

    if (tun.small_max >= 2) {
        PhaseScope ph(ctx, kPhCountSmall, s);
        TC_LAUNCH(ctx);
        int per_sm = 0;
        auto launch = [&](auto kern) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
            kern<<<(unsigned)(ns * std::max(per_sm, 1)), 256, 0, s>>>(a);
        };
        const bool step = tun.small_max > 8;  // longer lists: the branch-free merge step
        if (per_vertex) step ? launch(k_count_small<true, true>) : launch(k_count_small<true, false>);
        else step ? launch(k_count_small<false, true>) : launch(k_count_small<false, false>);
    }
    if (o->medge) {
        PhaseScope ph(ctx, kPhCountMerge, s);
        TC_LAUNCH(ctx);
        int per_sm = 0;
        if (per_vertex) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_merge<true>, 256, 0);
            k_count_merge<true><<<(unsigned)(ns * std::max(per_sm, 1)), 256, 0, s>>>(a, o->medge, &o->dc->n_merge_edges,
                                                                                     (unsigned long long)o->medge_cap);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_merge<false>, 256, 0);
            k_count_merge<false><<<(unsigned)(ns * std::max(per_sm, 1)), 256, 0, s>>>(a, o->medge, &o->dc->n_merge_edges,
                                                                                      (unsigned long long)o->medge_cap);
        }
    }
    if (tun.probe == kProbeBsearch) {
        e = per_vertex ? launch_tables<true, kProbeBsearch>(ctx, a, o, queues, ns, tun, s)
                       : launch_tables<false, kProbeBsearch>(ctx, a, o, queues, ns, tun, s);
    } else {
        e = per_vertex ? launch_tables<true, kProbeHash>(ctx, a, o, queues, ns, tun, s)
                       : launch_tables<false, kProbeHash>(ctx, a, o, queues, ns, tun, s);
    }
    if (e == cudaSuccess && t_rank) {
        PhaseScope ph(ctx, kPhCountInit, s);
        TC_LAUNCH(ctx);
        k_fold_rank_counts<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((o->n + 255) / 256, (int64_t)ns * 8)), 256, 0,
                             s>>>(o->n, o->perm, t_rank, per_vertex);
        e = cudaGetLastError();
    }
    dev_free(t_rank, s);
    dev_free(queues, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "count kernels");
    return TC_OK;
}

cudaError_t take_device_error(cudaStream_t s, unsigned* bits) {
    static const unsigned zero = 0u;
    unsigned h = 0u;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_tc_device_error, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbolAsync(g_tc_device_error, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *bits = h;
    return e;
}

cudaError_t peek_device_error_async(unsigned* h_pinned, cudaStream_t s) {
    if (!h_pinned) return cudaErrorInvalidValue;
    return cudaMemcpyFromSymbolAsync(h_pinned, g_tc_device_error, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
}

}  // namespace tc

extern "C" tc_status tc_check(tc_ctx* ctx, uint32_t* bits, void* stream) {
    if (!ctx) return TC_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    unsigned b = 0u;
    cudaError_t e = tc::take_device_error((cudaStream_t)stream, &b);
    if (bits) *bits = b;
    if (e != cudaSuccess) return tc::cuda_err(ctx, e, "tc_check");
    if (b) return tc::set_err(ctx, TC_ERR_DEVICE, "device check failed (check word 0x" + [](unsigned v) {
                                  char buf[16];
                                  snprintf(buf, sizeof buf, "%x", v);
                                  return std::string(buf);
                              }(b) + "): the results of the counts since the last check are not valid");
    return TC_OK;
}
