// k_list.cu -- neighbour-list rebuild: integer quantization, spatial sort
// into super-clusters, cluster-pair list with exact atom-pair masks, and the
// alchemical pair list.
//
// The listed pair set is defined on integer coordinates so that it is
// bit-exact and independent of floating-point contraction:
//   u = floor(frac(x L^-1) 2^24) (one rounded FP64 product),
//   d = ((u_i - u_j + 2^23) mod 2^24) - 2^23 per component,
//   listed iff D = |d|^2 < R = floor((r_list L^-1)^2 2^48), i < j, the pair is
//   not excluded, and at most one atom is alchemical.
// Each unordered pair appears in exactly one cluster-pair entry: the entry
// whose periodic shift equals the pair's minimum image, with the half-list
// rule (the j super-cluster less than half-way round the index circle from
// the i super-cluster, or the same one with a positive shift, or the same
// one with shift 0 and slot_i < slot_j).
#include "labf_internal.cuh"
#include "labf_launch.h"

namespace labf {

// -------------------------------------------------------------------------
// R1: quantize every real slot and count atoms per xy column
// -------------------------------------------------------------------------
__global__ void k_quantize(Dev d, int g0, int g1) {
    const int nthr = gridDim.x * blockDim.x;
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += nthr) {
        const int w = d.slot_walker[g];
        if (!la_in(d, w, d.n_walkers) || !d.rebuild[w]) continue;
        const int a = d.atom_of_slot[g];
        if (a < 0) continue;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        if (!la_in(d, a, S.n_atoms)) continue;
        const float4 x = d.xq[g];
        const uint32_t ux = quantize(x.x, S.box_inv), uy = quantize(x.y, S.box_inv),
                       uz = quantize(x.z, S.box_inv);
        const int cx = (int)(((unsigned long long)ux * (unsigned)S.ncx) >> 24);
        const int cy = (int)(((unsigned long long)uy * (unsigned)S.ncx) >> 24);
        const int c = cx + S.ncx * cy;
        if (!la_in(d, c, W.n_cols)) continue;
        d.t_uq[g] = make_int4((int)ux, (int)uy, (int)uz, a);
        d.t_col[g] = c;
        // one atomic per (walker, column) group of the warp's active lanes
        // (slots of a warp are spatially sorted, so most lanes share one)
        const int key = W.col_off + c;
        const unsigned grp = __match_any_sync(__activemask(), key);
        const int leader = __ffs(grp) - 1;
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == leader) base = atomicAdd(&d.col_count[key], __popc(grp));
        base = __shfl_sync(grp, base, leader);
        d.t_pos[g] = base + __popc(grp & ((1u << lane) - 1u));
    }
}

// R2: per walker (one warp), prefix sums of column counts and super-cluster
// counts, 32 columns per pass
__global__ void k_colscan(Dev d, int w0) {
    const int w = w0 + blockIdx.x;
    if (!d.rebuild[w]) return;
    const WalkerDev &W = d.walk[w];
    const int lane = threadIdx.x & 31;
    int acc = 0, sacc = 0;  // totals of the previous passes
    for (int c0 = 0; c0 < W.n_cols; c0 += 32) {
        const int c = c0 + lane;
        const int cnt = c < W.n_cols ? d.col_count[W.col_off + c] : 0;
        if (cnt > MAX_COL) set_status(d, LA_STATUS_COLUMN_OVERFLOW);
        const int nsc = (cnt + SC - 1) / SC;
        int a = cnt, b = nsc;  // inclusive warp scans
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) {
                a += ua;
                b += ub;
            }
        }
        if (c < W.n_cols) {
            d.col_start[W.col_off + c] = acc + a - cnt;
            d.col_sc[W.col_off + c] = sacc + b - nsc;
            d.col_nsc[W.col_off + c] = nsc;
        }
        acc += __shfl_sync(0xffffffffu, a, 31);
        sacc += __shfl_sync(0xffffffffu, b, 31);
    }
    if (lane == 0) {
        if (sacc > W.sc_cap) {
            set_status(d, LA_STATUS_LIST_OVERFLOW);
            sacc = W.sc_cap;
        }
        d.n_sc[w] = sacc;
    }
}

// R3: scatter slot ids into per-column buckets
__global__ void k_scatter(Dev d, int g0, int g1) {
    const int nthr = gridDim.x * blockDim.x;
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += nthr) {
        const int w = d.slot_walker[g];
        if (!la_in(d, w, d.n_walkers) || !d.rebuild[w] || d.atom_of_slot[g] < 0) continue;
        const WalkerDev &W = d.walk[w];
        const int c = d.t_col[g];
        if (!la_in(d, c, W.n_cols)) continue;
        const int p = d.col_start[W.col_off + c] + d.t_pos[g];
        if (!la_in(d, p, d.sys[W.sys].n_atoms)) continue;
        d.bucket[W.atom_base + p] = g;
    }
}

// R4: sort each column by (u_z, atom id) and cut it into super-clusters of 64
__global__ void __launch_bounds__(256) k_colsort(Dev d, int w0) {
    const int w = w0 + blockIdx.y;
    if (!d.rebuild[w]) return;
    const WalkerDev &W = d.walk[w];
    __shared__ unsigned long long key[MAX_COL];
    __shared__ int slot[MAX_COL];
    for (int c = blockIdx.x; c < W.n_cols; c += gridDim.x) {
        const int cnt0 = d.col_count[W.col_off + c];
        const int cnt = cnt0 > MAX_COL ? MAX_COL : cnt0;
        const int start = d.col_start[W.col_off + c];
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int g = d.bucket[W.atom_base + start + k];
            if (!la_in(d, g, d.n_slots)) {  // sorts last, written as padding
                key[k] = ~0ull;
                slot[k] = -1;
                continue;
            }
            const int4 u = d.t_uq[g];
            key[k] = ((unsigned long long)(unsigned)u.z << 32) | (unsigned)u.w;
            slot[k] = g;
        }
        __syncthreads();
        const int sc0 = W.sc_off + d.col_sc[W.col_off + c];
        const int nsc = d.col_nsc[W.col_off + c];
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const unsigned long long kk = key[k];
            int r = 0;
            for (int m = 0; m < cnt; ++m) r += key[m] < kk;
            const int s = sc0 + r / SC;
            if (s < W.sc_off + W.sc_cap) d.sc_member[(size_t)s * SC + (r % SC)] = slot[k];
        }
        for (int k = threadIdx.x; k < nsc * SC; k += blockDim.x) {
            const int s = sc0 + k / SC;
            if (k >= cnt && s < W.sc_off + W.sc_cap) d.sc_member[(size_t)s * SC + (k % SC)] = -1;
            if ((k % SC) == 0 && s < W.sc_off + W.sc_cap) d.sc_n[s] = min(SC, cnt - (k / SC) * SC);
        }
        __syncthreads();
        if (threadIdx.x == 0) d.col_count[W.col_off + c] = 0;  // ready for the next rebuild
    }
}

// R5: inside each super-cluster, four k-d splits (longest axis first, ranks
// by (coordinate, atom id), larger half first) give 16 leaves of <= 4 atoms;
// leaf k occupies slots 4k..4k+3.  Also the bounding boxes.  One warp per
// super-cluster.
__global__ void __launch_bounds__(128) k_kdsplit(Dev d, int w0, int w1) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __shared__ int sx[4][SC], sy[4][SC], sz[4][SC], sa[4][SC], sg[4][SC], sslot[4][SC];
    const int nwarp = gridDim.x * (blockDim.x >> 5);
    const int s_begin = d.walk[w0].sc_off, s_end = d.walk[w1 - 1].sc_off + d.walk[w1 - 1].sc_cap;
    for (int s = s_begin + blockIdx.x * (blockDim.x >> 5) + wib; s < s_end; s += nwarp) {
        int lo = w0, hi = w1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (d.walk[mid].sc_off <= s) lo = mid; else hi = mid - 1;
        }
        const int w = lo;
        if (!d.rebuild[w]) continue;
        const WalkerDev &W = d.walk[w];
        const int s_local = s - W.sc_off;
        if (s_local >= d.n_sc[w]) continue;
        const int n = d.sc_n[s];
        for (int k = lane; k < SC; k += 32) {
            int g = k < n ? d.sc_member[(size_t)s * SC + k] : -1;
            if (g >= 0 && !la_in(d, g, d.n_slots)) g = -1;
            if (g >= 0) {
                const int4 u = d.t_uq[g];
                sx[wib][k] = u.x; sy[wib][k] = u.y; sz[wib][k] = u.z; sa[wib][k] = u.w;
            } else {
                sa[wib][k] = -1;
            }
            sslot[wib][k] = g;
            sg[wib][k] = 0;
        }
        __syncwarp();
        // leaf index by four binary splits
        for (int level = 0; level < 4; ++level) {
            // extent and size of every group of this level by warp reductions;
            // each lane keeps those of its two atoms' groups
            int ext[2][3] = {{0, 0, 0}, {0, 0, 0}}, cnts[2] = {0, 0};
            {
                const int ga = lane < n ? sg[wib][lane] : -1;
                const int gb = lane + 32 < n ? sg[wib][lane + 32] : -1;
                const int xa[3] = {sx[wib][lane], sy[wib][lane], sz[wib][lane]};
                const int xb[3] = {sx[wib][lane + 32], sy[wib][lane + 32], sz[wib][lane + 32]};
                for (int g = 0; g < (1 << level); ++g) {
                    const bool ia = ga == g, ib = gb == g;
                    const int c = __reduce_add_sync(0xffffffffu, (int)ia + (int)ib);
                    for (int q = 0; q < 3; ++q) {
                        const int lo = __reduce_min_sync(0xffffffffu, min(ia ? xa[q] : (1 << 30), ib ? xb[q] : (1 << 30)));
                        const int hi = __reduce_max_sync(0xffffffffu, max(ia ? xa[q] : -1, ib ? xb[q] : -1));
                        if (ia) ext[0][q] = hi - lo;
                        if (ib) ext[1][q] = hi - lo;
                    }
                    if (ia) cnts[0] = c;
                    if (ib) cnts[1] = c;
                }
            }
            int newg[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = lane + 32 * h;
                newg[h] = sg[wib][k];
                if (k >= n) continue;
                const int gid = sg[wib][k];
                const int cnt = cnts[h];
                // longest axis, the first of equal ones
                int ax = 0, eb = ext[h][0];
                if (ext[h][1] > eb) {
                    ax = 1;
                    eb = ext[h][1];
                }
                if (ext[h][2] > eb) ax = 2;
                const int *co = ax == 0 ? sx[wib] : (ax == 1 ? sy[wib] : sz[wib]);
                const long long mykey = ((long long)co[k] << 32) | (unsigned)sa[wib][k];
                int r = 0;
                for (int m = 0; m < n; ++m) {
                    if (sg[wib][m] != gid) continue;
                    const long long km = ((long long)co[m] << 32) | (unsigned)sa[wib][m];
                    r += km < mykey;
                }
                newg[h] = 2 * gid + (r >= (cnt + 1) / 2 ? 1 : 0);
            }
            __syncwarp();
            sg[wib][lane] = newg[0];
            sg[wib][lane + 32] = newg[1];
            __syncwarp();
        }
        // final position inside the leaf: rank by atom id
        int pos[2];
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            pos[h] = -1;
            if (k >= n) continue;
            int r = 0;
            for (int m = 0; m < n; ++m) r += (sg[wib][m] == sg[wib][k]) && (sa[wib][m] < sa[wib][k]);
            pos[h] = sg[wib][k] * JC + r;
        }
        // new layout: t_old[new slot] = old slot (-1 for padding)
        const int gbase = W.slot_off + s_local * SC;
        d.t_old[gbase + lane] = -1;
        d.t_old[gbase + lane + 32] = -1;
        __syncwarp();
        for (int h = 0; h < 2; ++h)
            if (pos[h] >= 0) d.t_old[gbase + pos[h]] = sslot[wib][lane + 32 * h];
        __syncwarp();
        // bounding boxes (integer, real atoms only): j-clusters, i-clusters, super-cluster
        if (lane < NJC + NIC + 1) {
            int first, last;
            if (lane < NJC) { first = lane; last = lane; }
            else if (lane < NJC + NIC) { first = 2 * (lane - NJC); last = first + 1; }
            else { first = 0; last = NJC - 1; }
            int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-(1 << 30), -(1 << 30), -(1 << 30)}, cnt = 0;
            for (int m = 0; m < n; ++m) {
                const int leaf = sg[wib][m];
                if (leaf < first || leaf > last) continue;
                ++cnt;
                mn[0] = min(mn[0], sx[wib][m]); mx[0] = max(mx[0], sx[wib][m]);
                mn[1] = min(mn[1], sy[wib][m]); mx[1] = max(mx[1], sy[wib][m]);
                mn[2] = min(mn[2], sz[wib][m]); mx[2] = max(mx[2], sz[wib][m]);
            }
            int4 *dst;
            if (lane < NJC) dst = d.bb_jc + 2 * ((size_t)s * NJC + lane);
            else if (lane < NJC + NIC) dst = d.bb_ic + 2 * ((size_t)s * NIC + (lane - NJC));
            else dst = d.bb_sc + 2 * (size_t)s;
            dst[0] = make_int4(mn[0], mn[1], mn[2], cnt);
            dst[1] = make_int4(mx[0], mx[1], mx[2], 0);
        }
        __syncwarp();
    }
}

// R6: gather the state into the new slot order (scratch buffers)
__global__ void k_permute_gather(Dev d, int g0, int g1) {
    const int nthr = gridDim.x * blockDim.x;
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += nthr) {
        const int w = d.slot_walker[g];
        if (!d.rebuild[w]) continue;
        const WalkerDev &W = d.walk[w];
        const int local = g - W.slot_off;
        const int s_local = local / SC;
        int old = -1;
        if (s_local < d.n_sc[w]) old = d.t_old[g];
        if (old >= 0 && !la_in(d, old, d.n_slots)) old = -1;
        if (old >= 0) {
            d.t_xq[g] = d.xq[old];
            d.t_vv[g] = d.vv[old];
            d.uq[g] = d.t_uq[old];
        } else {
            // padding: park on a real atom of the same super-cluster (finite,
            // never listed) or, for unused super-clusters, at the origin
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            if (s_local < d.n_sc[w]) {
                const int first = d.sc_member[(size_t)(W.sc_off + s_local) * SC];
                if (first >= 0 && la_in(d, first, d.n_slots)) p = d.xq[first];
            }
            p.w = 0.f;
            d.t_xq[g] = p;
            d.t_vv[g] = make_float4(0.f, 0.f, 0.f, 0.f);
            d.uq[g] = make_int4(0, 0, 0, -1);
        }
    }
}

// R7: write the new layout back and refresh per-slot parameters
__global__ void k_permute_scatter(Dev d, int g0, int g1) {
    const int nthr = gridDim.x * blockDim.x;
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += nthr) {
        const int w = d.slot_walker[g];
        if (!d.rebuild[w]) continue;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        int a = d.uq[g].w;
        if (a >= 0 && !la_in(d, a, S.n_atoms)) a = -1;
        float4 x = d.t_xq[g];
        // wrap into [0, L) (the list built from this layout assumes it)
        x.x -= S.boxf * floorf(x.x * S.box_invf);
        x.y -= S.boxf * floorf(x.y * S.box_invf);
        x.z -= S.boxf * floorf(x.z * S.box_invf);
        d.vv[g] = d.t_vv[g];
        d.atom_of_slot[g] = a;
        if (a >= 0) {
            const float4 ap = d.aparam_mut[S.atom_off + a];
            x.w = ap.x;
            d.lj[g] = make_float2(ap.y, ap.z);
            d.im[g] = make_float2(ap.w, d.anoise[S.atom_off + a]);
            d.slot_of_atom[W.atom_base + a] = g;
            d.smeta[g] = make_int2(d.agroup[S.atom_off + a], (int)d.aalch[S.atom_off + a]);
            d.sexcl[g] = d.aexcl[S.atom_off + a];
        } else {
            d.lj[g] = make_float2(0.f, 0.f);
            d.im[g] = make_float2(0.f, 0.f);
            d.smeta[g] = make_int2(-1, 1);
            d.sexcl[g] = make_int4(-1, -1, -1, -1);
        }
        d.xq[g] = x;
        d.xref[g] = x;
    }
}

// -------------------------------------------------------------------------
// R8: cluster-pair list.  One warp per work item (super-cluster S, run of
// LB_CHUNK candidate column slots k): the k-th column (with its periodic
// image) within reach of S's box.
// For every candidate super-cluster T of that column (cyclic half rule) T's
// 64 slots are staged in shared memory, the 16 x 8 (j-cluster, i-cluster)
// box tests run lane-parallel, and for each passing pair of clusters lane
// (ia, jb) = (lane & 7, lane >> 3) tests the atom pair (8 ic + ia of S,
// 4 jc + jb of T) exactly.  Entries go to the (S, k) sub-list; R8b
// concatenates the sub-lists of S in k order.
// -------------------------------------------------------------------------
__device__ __forceinline__ long long bb_dist2(const int4 &alo, const int4 &ahi, const int4 &blo,
                                              const int4 &bhi, int sx, int sy, int sz) {
    long long dx = max(0, max(blo.x + sx - ahi.x, alo.x - (bhi.x + sx)));
    long long dy = max(0, max(blo.y + sy - ahi.y, alo.y - (bhi.y + sy)));
    long long dz = max(0, max(blo.z + sz - ahi.z, alo.z - (bhi.z + sz)));
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// nonbonded exclusion of two real atoms (group, then extra partner lists)
__device__ __forceinline__ bool excluded_meta(int a, int2 ma, int4 ea, int b, int2 mb, int4 eb) {
    if (ma.x >= 0 && ma.x == mb.x) return true;
    if (ea.x == b || ea.y == b || ea.z == b || ea.w == b) return true;
    return eb.x == a || eb.y == a || eb.z == a || eb.w == a;
}

constexpr int LB_WARPS = 4;
// Staged slots: coordinates, and in .w a code = exclusion group (bits 0-29)
// | EXTRA_FLAG when the slot has extra excluded partners.  Slots without
// normal pairs (padding, alchemical) sit at FAR_I on the i side and FAR_J on
// the j side (|d| >= 2^30 - 2^24 per component, so D >= R for every list
// radius, and 3 (2^30 + 2^24)^2 < 2^63); "no group" has a different code on
// each side, so that one compare decides the group test.
constexpr int FAR_I = 1 << 29, FAR_J = -(1 << 29);
constexpr int GROUP_MASK = 0x3fffffff, EXTRA_FLAG = 0x40000000;
constexpr int NO_GROUP_I = 0x3fffffff, NO_GROUP_J = 0x3ffffffe;

__device__ __forceinline__ int slot_code(int2 m, int4 e, bool i_side) {
    const int g = m.x >= 0 ? m.x : (i_side ? NO_GROUP_I : NO_GROUP_J);
    return g | ((e.x & e.y & e.z & e.w) != -1 ? EXTRA_FLAG : 0);
}

// extra excluded partners of two real atoms (atom ids and lists from memory)
__device__ __forceinline__ bool excluded_extra(const Dev &d, int gi, int gj) {
    const int a = d.uq[gi].w, b = d.uq[gj].w;
    const int4 ea = d.sexcl[gi], eb = d.sexcl[gj];
    if (ea.x == b || ea.y == b || ea.z == b || ea.w == b) return true;
    return eb.x == a || eb.y == a || eb.z == a || eb.w == a;
}

// lane (ia, jb)'s mask byte of one candidate j-cluster: bit ic set when the
// pair (8 ic + ia of S, slot sj of T) is listed.  SELF: S and T are the
// same super-cluster with shift 0, where only slot_i < slot_j is listed.
template <bool SELF>
__device__ __forceinline__ unsigned tile_masks(const int4 *su, unsigned cand, int ia, int sj, int ujx, int ujy,
                                               int ujz, int cj, long long R, const Dev &d, int gS, int gT) {
    unsigned lbyte = 0;
    for (unsigned m = cand; m; m &= m - 1u) {  // candidate i-clusters, ascending
        const int ic = __ffs(m) - 1;
        const int si = ic * IC + ia;
        const int4 ui = su[si];
        // D < R implies every component lies in (-2^23, 2^23) (R <= 2^46
        // because L >= 2 r_list), i.e. this shift is the minimum image
        const int dx = ujx - ui.x, dy = ujy - ui.y, dz = ujz - ui.z;
        bool ok = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz < R && ((ui.w ^ cj) & GROUP_MASK) != 0;
        if (SELF) ok = ok && si < sj;
        if (ok && ((ui.w | cj) & EXTRA_FLAG)) ok = !excluded_extra(d, gS + si, gT + sj);
        lbyte |= (unsigned)ok << ic;
    }
    return lbyte;
}
constexpr int LB_CHUNK = 1;  // candidate-column slots per work item

// work items (S, run of LB_CHUNK candidate-column slots) of the walkers that
// rebuild are handed out by a global counter (counters[8]); the last warp
// out (counters[9]) resets both for the next launch
constexpr int CTR_LB_ITEM = 8, CTR_LB_DONE = 9;

__global__ void __launch_bounds__(LB_WARPS * 32, 8) k_listbuild(Dev d, int w0, int w1) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int ia = lane & 7, jb = lane >> 3;
    __shared__ int4 s_u[LB_WARPS][SC], t_u[LB_WARPS][SC];
    __shared__ int4 s_bb[LB_WARPS][2 * NIC + 2], t_bb[LB_WARPS][2 * NJC];
    __shared__ int s_pre[LA_MAX_WALKERS_PER_LAUNCH + 1], s_wk[LA_MAX_WALKERS_PER_LAUNCH];
    __shared__ int s_nw;
    const int nchunk = (d.ncs + LB_CHUNK - 1) / LB_CHUNK;
    // prefix of the work items over the walkers that rebuild (their actual
    // super-clusters only), so that walkers without a rebuild cost nothing
    if (wib == 0) {
        int acc = 0, nw = 0;
        for (int base = w0; base < w1; base += 32) {
            const int w = base + lane;
            const bool on = w < w1 && d.rebuild[w] != 0;
            int units = on ? d.n_sc[w] * nchunk : 0, rank = on ? 1 : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int a = __shfl_up_sync(0xffffffffu, units, o), b = __shfl_up_sync(0xffffffffu, rank, o);
                if (lane >= o) {
                    units += a;
                    rank += b;
                }
            }
            if (on) {
                s_pre[nw + rank - 1] = acc + units - d.n_sc[w] * nchunk;
                s_wk[nw + rank - 1] = w;
            }
            acc += __shfl_sync(0xffffffffu, units, 31);
            nw += __shfl_sync(0xffffffffu, rank, 31);
        }
        if (lane == 0) {
            s_pre[nw] = acc;
            s_nw = nw;
        }
    }
    __syncthreads();
    const int nw_on = s_nw;
    const long long total = s_pre[nw_on];
    for (;;) {
        long long idx = 0;
        if (lane == 0) idx = (long long)atomicAdd(&d.counters[CTR_LB_ITEM], 1ull);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= total) break;
        int lo = 0, hi = nw_on - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= idx) lo = mid; else hi = mid - 1;
        }
        const int w = s_wk[lo];
        const int local = (int)(idx - s_pre[lo]);
        const int s = d.walk[w].sc_off + local / nchunk;
        const int k0 = (local % nchunk) * LB_CHUNK;
        for (int kslot = k0; kslot < k0 + LB_CHUNK && kslot < d.ncs; ++kslot) {
            const WalkerDev &W = d.walk[w];
            const SysDev &S = d.sys[W.sys];
            const int S_loc = s - W.sc_off;
            const int nsc = d.n_sc[w];
            const size_t sub = (size_t)s * d.ncs + kslot;
            if (kslot >= S.cspan * S.cspan) {
                if (lane == 0) d.sub_n[sub] = 0;
                continue;
            }
            const int4 slo = d.bb_sc[2 * (size_t)s], shi = d.bb_sc[2 * (size_t)s + 1];
            const int ncx = S.ncx;
            const int cx0 = (int)(((long long)(slo.x - S.Rq) * ncx) >> 24);
            const int cx1 = (int)(((long long)(shi.x + S.Rq) * ncx) >> 24);
            const int cy0 = (int)(((long long)(slo.y - S.Rq) * ncx) >> 24);
            const int cy1 = (int)(((long long)(shi.y + S.Rq) * ncx) >> 24);
            const int cx = cx0 + kslot % S.cspan, cy = cy0 + kslot / S.cspan;
            if (cx > cx1 || cy > cy1) {
                if (lane == 0) d.sub_n[sub] = 0;
                continue;
            }
            if (kslot == 0 && lane == 0 && (cx1 - cx0 >= S.cspan || cy1 - cy0 >= S.cspan))
                set_status(d, LA_STATUS_LIST_OVERFLOW);  // cannot happen for boxes inside a column
            const int gS = W.slot_off + S_loc * SC;
            __syncwarp();
            // staged: coordinates (FAR_I for a slot without normal pairs) and
            // the slot code (exclusion group, extra-partner flag)
            for (int k = lane; k < SC; k += 32) {
                int4 u = d.uq[gS + k];
                const int2 m = d.smeta[gS + k];
                const int4 e = d.sexcl[gS + k];
                if (m.y || u.w < 0) u.x = u.y = u.z = FAR_I;
                u.w = slot_code(m, e, true);
                s_u[wib][k] = u;
            }
            if (lane < 2 * NIC) s_bb[wib][lane] = d.bb_ic[2 * (size_t)s * NIC + lane];
            __syncwarp();
            const long long R = S.R;
            const int U = 1 << 24;
            const int ty = floordiv(cy, ncx), wy = cy - ty * ncx;
            const int tx = floordiv(cx, ncx), wx = cx - tx * ncx;
            const int col = wx + ncx * wy;
            if (!la_in(d, col, W.n_cols)) {
                if (lane == 0) d.sub_n[sub] = 0;
                continue;
            }
            const int t0 = d.col_sc[W.col_off + col], tn = d.col_nsc[W.col_off + col];
            int nent = 0;
            const size_t ebase = sub * d.sub_cap;
            const int t_end = min(t0 + tn, nsc);
            // the column's super-clusters 32 at a time: lane l tests T = tb + l
            // (half-list rule, then its box against S's box for the three z
            // shifts); the warp then visits the T with a shift in range in
            // ascending order
            for (int tb = t0; tb < t_end; tb += 32) {
                unsigned zp_l = 0;  // z shifts whose super-cluster boxes are in range
                {
                    const int T_loc = tb + lane;
                    bool partner = T_loc < t_end;
                    // cyclic half list over super-clusters: T is S's partner when it
                    // lies less than half-way round the index circle
                    if (partner && T_loc != S_loc) {
                        const int del = T_loc > S_loc ? T_loc - S_loc : T_loc - S_loc + nsc;
                        partner = !(2 * del > nsc || (2 * del == nsc && T_loc < S_loc));
                    }
                    if (partner) {
                        const int t = W.sc_off + T_loc;
                        const int4 tlo = d.bb_sc[2 * (size_t)t], thi = d.bb_sc[2 * (size_t)t + 1];
                        if (tlo.w != 0) {
                            for (int tz = -1; tz <= 1; ++tz) {
                                if (T_loc == S_loc && (tx < 0 || (tx == 0 && (ty < 0 || (ty == 0 && tz < 0))))) continue;
                                if (bb_dist2(slo, shi, tlo, thi, tx * U, ty * U, tz * U) < R) zp_l |= 1u << (tz + 1);
                            }
                        }
                    }
                }
                for (unsigned tmask = __ballot_sync(0xffffffffu, zp_l != 0u); tmask; tmask &= tmask - 1u) {
                    const int tl = __ffs(tmask) - 1;
                    const int T_loc = tb + tl;
                    const unsigned zpass = __shfl_sync(0xffffffffu, zp_l, tl);
                    const int t = W.sc_off + T_loc;
                    const int gT = W.slot_off + T_loc * SC;
                    __syncwarp();
                    for (int k = lane; k < SC; k += 32) {
                        int4 u = d.uq[gT + k];
                        const int2 m = d.smeta[gT + k];
                        const int4 e = d.sexcl[gT + k];
                        if (m.y || u.w < 0) u.x = u.y = u.z = FAR_J;
                        u.w = slot_code(m, e, false);
                        t_u[wib][k] = u;
                    }
                    t_bb[wib][lane] = d.bb_jc[2 * (size_t)t * NJC + lane];
                    __syncwarp();
                    for (int tz = -1; tz <= 1; ++tz) {
                        if (!(zpass & (1u << (tz + 1)))) continue;
                        const int shx = tx * U, shy = ty * U, shz = tz * U;
                        const bool self0 = (T_loc == S_loc) && tx == 0 && ty == 0 && tz == 0;
                        const int shift_bits = (tx + 1) | ((ty + 1) << 2) | ((tz + 1) << 4);
                        // lane-parallel box tests of the 128 (jc, ic) combinations:
                        // bit (jc & 3) * 8 + ic of word jc >> 2
                        unsigned cm0, cm1, cm2, cm3;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = lane + 32 * q, jc = c >> 3, ic = c & 7;
                            const int4 jlo = t_bb[wib][2 * jc], jhi = t_bb[wib][2 * jc + 1];
                            const int4 ilo = s_bb[wib][2 * ic], ihi = s_bb[wib][2 * ic + 1];
                            const bool ok = jlo.w > 0 && ilo.w > 0 && bb_dist2(ilo, ihi, jlo, jhi, shx, shy, shz) < R;
                            const unsigned b = __ballot_sync(0xffffffffu, ok);
                            if (q == 0) cm0 = b; else if (q == 1) cm1 = b; else if (q == 2) cm2 = b; else cm3 = b;
                        }
                        // j-clusters with at least one candidate i-cluster, ascending
                        // (a non-zero byte of a word -> one bit: the byte flags
                        // 0x01 at bits 0, 8, 16, 24 times 0x01020408 land at
                        // bits 24-27 without carries)
                        const auto nib = [](unsigned w) {
                            return ((__vcmpne4(w, 0u) & 0x01010101u) * 0x01020408u) >> 24;
                        };
                        unsigned jmask = nib(cm0) | (nib(cm1) << 4) | (nib(cm2) << 8) | (nib(cm3) << 12);
                        for (; jmask; jmask &= jmask - 1u) {
                            const int jc = __ffs(jmask) - 1;
                            const unsigned cw = jc < 8 ? (jc < 4 ? cm0 : cm1) : (jc < 12 ? cm2 : cm3);
                            const unsigned cand = (cw >> ((jc & 3) * 8)) & 0xffu;
                            const int4 uj = t_u[wib][jc * JC + jb];
                            const int ujx = uj.x + shx, ujy = uj.y + shy, ujz = uj.z + shz;
                            const unsigned lbyte =
                                self0 ? tile_masks<true>(s_u[wib], cand, ia, jc * JC + jb, ujx, ujy, ujz, uj.w, R, d, gS, gT)
                                      : tile_masks<false>(s_u[wib], cand, ia, jc * JC + jb, ujx, ujy, ujz, uj.w, R, d, gS, gT);
                            const unsigned imask = __reduce_or_sync(0xffffffffu, lbyte);
                            if (imask) {
                                if (nent < d.sub_cap) {
                                    const size_t e = ebase + nent;
                                    // i-cluster mask twice: bits 8-15 are pruned by the batched
                                    // step, bits 16-23 keep the listed set
                                    if (lane == 0)
                                        d.sub_hdr[e] = make_int2(gT + jc * JC, shift_bits | (int)(imask << 8) | (int)(imask << 16));
                                    d.sub_lb[32 * e + lane] = (unsigned char)lbyte;
                                } else if (lane == 0) {
                                    set_status(d, LA_STATUS_LIST_OVERFLOW);
                                }
                                ++nent;
                            }
                        }
                    }
                }
            }
            if (lane == 0) d.sub_n[sub] = min(nent, d.sub_cap);
            __syncwarp();
        }
    }
    // the last warp out resets the work counters for the next launch
    if (lane == 0) {
        __threadfence();
        const unsigned long long done = atomicAdd(&d.counters[CTR_LB_DONE], 1ull);
        if (done == (unsigned long long)gridDim.x * LB_WARPS - 1ull) {
            d.counters[CTR_LB_ITEM] = 0ull;
            d.counters[CTR_LB_DONE] = 0ull;
            __threadfence();
        }
    }
}

// R8b: concatenate the sub-lists of each super-cluster in column-slot order
__global__ void __launch_bounds__(128) k_listcompact(Dev d, int w0, int w1) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __shared__ int s_off[4][32];
    const int nwarp = gridDim.x * (blockDim.x >> 5);
    const int s_begin = d.walk[w0].sc_off, s_end = d.walk[w1 - 1].sc_off + d.walk[w1 - 1].sc_cap;
    for (int s = s_begin + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < s_end; s += nwarp) {
        int lo = w0, hi = w1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (d.walk[mid].sc_off <= s) lo = mid; else hi = mid - 1;
        }
        if (!d.rebuild[lo]) continue;
        if (s - d.walk[lo].sc_off >= d.n_sc[lo]) {  // capacity slot without a super-cluster
            if (lane == 0) d.sc_nent[s] = 0;
            continue;
        }
        const size_t ebase = (size_t)s * d.ent_cap;
        int n = 0;
        // 32 sub-lists at a time: their sizes by one load per lane and a warp
        // scan, then every entry of the 32 copied by a flat lane loop (the
        // sub-list of flat index f found by binary search over the offsets)
        for (int k0 = 0; k0 < d.ncs; k0 += 32) {
            const int k = k0 + lane;
            const int m = k < d.ncs ? d.sub_n[(size_t)s * d.ncs + k] : 0;
            int incl = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            s_off[wib][lane] = incl - m;
            __syncwarp();
            for (int f = lane; f < tot && n + f < d.ent_cap; f += 32) {
                int lo = 0, hi = 31;  // the last sub-list starting at or before f
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[wib][mid] <= f) lo = mid; else hi = mid - 1;
                }
                const size_t src = ((size_t)s * d.ncs + k0 + lo) * d.sub_cap + (f - s_off[wib][lo]);
                const size_t dst = ebase + n + f;
                d.ent_hdr[dst] = d.sub_hdr[src];
                const uint4 *ps = reinterpret_cast<const uint4 *>(d.sub_lb + 32 * src);
                uint4 *pd = reinterpret_cast<uint4 *>(d.ent_lb + 32 * dst);
                pd[0] = ps[0];
                pd[1] = ps[1];
            }
            __syncwarp();
            n += tot;
        }
        if (n > d.ent_cap && lane == 0) set_status(d, LA_STATUS_LIST_OVERFLOW);
        if (lane == 0) d.sc_nent[s] = min(n, d.ent_cap);
    }
}

// -------------------------------------------------------------------------
// R9: alchemical list: one block per (walker, alchemical atom).  Super-cluster
// boxes are tested lane-parallel; the 64 slots of each box in range are then
// tested exactly (two per lane) by the block's warps in turn, and the hits
// are written in super-cluster and slot order (deterministic output order).
// -------------------------------------------------------------------------
constexpr int AL_WARPS = 4;

__global__ void __launch_bounds__(AL_WARPS * 32) k_alchlist(Dev d, int w0, int w1, int a0, int a1) {
    // one block per (walker, alchemical atom); the super-clusters are box
    // tested one per thread, 128 per round, the near ones compacted in
    // ascending order and tested slot by slot by the block's warps in turn,
    // and warp 0 writes the hits in (super-cluster, slot) order
    constexpr int NT = AL_WARPS * 32;
    __shared__ unsigned long long okm[NT];
    __shared__ int near_sc[NT];
    __shared__ int wcnt[AL_WARPS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int it = a0 + blockIdx.x; it < a1; it += gridDim.x) {
        int lo = w0, hi = w1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (d.walk[mid].alch_base <= it) lo = mid; else hi = mid - 1;
        }
        const int w = lo;
        if (!d.rebuild[w]) continue;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        const int r = it - W.alch_base;
        const int a = d.alch_atoms[S.alch_off + r];
        if (!la_in(d, a, S.n_atoms)) continue;
        const int ga = d.slot_of_atom[W.atom_base + a];
        if (!la_in(d, ga, d.n_slots)) continue;
        const int4 ua = d.uq[ga];
        const int2 ma = d.smeta[ga];
        const int4 ea = d.sexcl[ga];
        const int U = 1 << 24;
        int cnt = 0;
        const int nsc = d.n_sc[w];
        int *out = d.alch_slot + (size_t)it * d.alch_cap;
        for (int b0 = 0; b0 < nsc; b0 += NT) {
            // super-cluster box within the list radius of the atom (any image)
            bool near = false;
            if (b0 + (int)threadIdx.x < nsc) {
                const size_t t = (size_t)(W.sc_off + b0 + threadIdx.x);
                const int4 tlo = d.bb_sc[2 * t], thi = d.bb_sc[2 * t + 1];
                if (tlo.w > 0) {
                    long long D = 0;
                    const int uc[3] = {ua.x, ua.y, ua.z};
                    const int lc[3] = {tlo.x, tlo.y, tlo.z}, hc[3] = {thi.x, thi.y, thi.z};
                    for (int c = 0; c < 3; ++c) {
                        long long best = -1;
                        for (int sh = -1; sh <= 1; ++sh) {
                            const long long gap = max(0, max(lc[c] + sh * U - uc[c], uc[c] - (hc[c] + sh * U)));
                            if (best < 0 || gap < best) best = gap;
                        }
                        D += best * best;
                    }
                    near = D < S.R;
                }
            }
            // compaction in ascending order: warp counts, then offsets
            const unsigned nm = __ballot_sync(0xffffffffu, near);
            if (lane == 0) wcnt[wib] = __popc(nm);
            __syncthreads();
            int off = 0, nn = 0;
            for (int q = 0; q < AL_WARPS; ++q) {
                off += q < wib ? wcnt[q] : 0;
                nn += wcnt[q];
            }
            if (near) near_sc[off + __popc(nm & ((1u << lane) - 1u))] = b0 + threadIdx.x;
            __syncthreads();
            for (int kk = wib; kk < nn; kk += AL_WARPS) {
                const int gbase = W.slot_off + near_sc[kk] * SC;
                unsigned bits[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int g = gbase + lane + 32 * h;
                    const int4 ub = d.uq[g];
                    const int2 mb = d.smeta[g];
                    bool ok = false;
                    if (ub.w >= 0 && !mb.y) {
                        const long long dx = torus_delta(ub.x, ua.x), dy = torus_delta(ub.y, ua.y),
                                        dz = torus_delta(ub.z, ua.z);
                        ok = dx * dx + dy * dy + dz * dz < S.R && !excluded_meta(a, ma, ea, ub.w, mb, d.sexcl[g]);
                    }
                    bits[h] = __ballot_sync(0xffffffffu, ok);
                }
                if (lane == 0) okm[kk] = ((unsigned long long)bits[1] << 32) | bits[0];
            }
            __syncthreads();
            if (wib == 0) {
                for (int kk = 0; kk < nn; ++kk) {
                    const int gbase = W.slot_off + near_sc[kk] * SC;
                    const unsigned long long om = okm[kk];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const unsigned mh = h ? (unsigned)(om >> 32) : (unsigned)om;
                        const int pos = cnt + __popc(mh & ((1u << lane) - 1u));
                        if (((mh >> lane) & 1u) && pos < d.alch_cap) out[pos] = gbase + lane + 32 * h;
                        cnt += __popc(mh);
                    }
                }
            }
            __syncthreads();
        }
        if (wib == 0) {
            if (cnt > d.alch_cap) {
                if (lane == 0) set_status(d, LA_STATUS_ALCH_OVERFLOW);
                cnt = d.alch_cap;
            }
            if (lane == 0) d.alch_cnt[it] = cnt;
        }
    }
}

// -------------------------------------------------------------------------
// R10: pair-kernel work items (chunks of `chunk` entries of one
// super-cluster), per walker; clears the rebuild flag.  In the batched step
// (prune_fresh) a walker with pruning on has its fresh list pruned by this
// step's pair pass.
// -------------------------------------------------------------------------
__global__ void k_items(Dev d, int w0, int prune_fresh) {
    const int w = w0 + blockIdx.x;
    if (!d.rebuild[w]) return;
    const WalkerDev &W = d.walk[w];
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int nsc = d.n_sc[w];
    for (int base = 0; base < nsc; base += blockDim.x) {
        const int sl = base + threadIdx.x;
        const int ne = sl < nsc ? d.sc_nent[W.sc_off + sl] : 0;
        const int nch = (ne + d.chunk - 1) / d.chunk;
        // block exclusive scan of nch
        int v = nch;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const int excl = carry + v - nch + (wid > 0 ? wsum[wid - 1] : 0);
        for (int c = 0; c < nch; ++c) {
            const int item = excl + c;
            if (item < W.item_cap) {
                const int e0 = c * d.chunk, e1 = min(ne, e0 + d.chunk);
                d.items[W.item_base + item] = make_int4(W.sc_off + sl, e0, e1, w);
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + nch;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (carry > W.item_cap) set_status(d, LA_STATUS_LIST_OVERFLOW);
        d.n_items[w] = min(carry, W.item_cap);
        d.rebuild[w] = 0;
        d.near[w] = 0;
        if (prune_fresh && d.sys[W.sys].prune_disp2 > 0.f) d.prune_now[w] = d.step[w] + 1ull;
        atomicAdd(&d.counters[0], 1ull);
    }
}

// -------------------------------------------------------------------------
// gate of the batched step, after the integrator: a walker whose pruning was
// requested is re-pruned by this step's pair pass (prune_now = 1 + step
// counter; the next integrator step takes the positions it starts from as the
// walker's new reference).  When some walker must rebuild, the walkers whose
// systems are due soon (near flags) join it (coalescing).  Inside a CUDA
// graph one thread also sets the step's conditional handle to "some walker
// must rebuild", so that the graph skips the list kernels otherwise; such
// steps are counted in counters[6].
// -------------------------------------------------------------------------
__device__ __forceinline__ void coalesce_rebuilds(const Dev &d, int w0, int w1, int any) {
    if (!any) return;
    for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x)
        if (d.near[w]) d.rebuild[w] = 1;
}

__global__ void k_gate(Dev d, int w0, int w1, cudaGraphConditionalHandle handle, int conditional) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        const int p = d.prune[w];
        d.prune_now[w] = p ? d.step[w] + 1ull : 0ull;
        if (p) {
            d.prune[w] = 0;
            atomicAdd(&d.counters[10], 1ull);
        }
        if (d.rebuild[w]) any = 1;
    }
    __syncthreads();
    coalesce_rebuilds(d, w0, w1, any);
    if (conditional && threadIdx.x == 0) {
        cudaGraphSetConditional(handle, any ? 1u : 0u);
        if (any) atomicAdd(&d.counters[6], 1ull);
    }
}

void launch_gate(const Dev &d, int w0, int w1, cudaGraphConditionalHandle handle, bool conditional,
                 cudaStream_t s) {
    k_gate<<<1, 256, 0, s>>>(d, w0, w1, handle, conditional ? 1 : 0);
}

// the one-walker-per-launch form's coalescing (no pruning there)
__global__ void k_coalesce(Dev d, int w0, int w1) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x)
        if (d.rebuild[w]) any = 1;
    __syncthreads();
    coalesce_rebuilds(d, w0, w1, any);
}

void launch_coalesce(const Dev &d, int w0, int w1, cudaStream_t s) { k_coalesce<<<1, 256, 0, s>>>(d, w0, w1); }

// -------------------------------------------------------------------------
// host launcher of the whole rebuild chain (every kernel exits early for
// walkers whose rebuild flag is clear)
// -------------------------------------------------------------------------
void launch_rebuild(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s, bool batched) {
    const int g0 = hv.slot_off[w0], g1 = hv.slot_off[w1 - 1] + hv.slot_cap[w1 - 1];
    int sb = (g1 - g0 + 255) / 256;
    sb = sb < 1 ? 1 : (sb > hv.n_sm * 8 ? hv.n_sm * 8 : sb);
    const int nw = w1 - w0;
    int max_cols = 1;
    for (int w = w0; w < w1; ++w) max_cols = hv.n_cols[w] > max_cols ? hv.n_cols[w] : max_cols;
    int nsc = 0;
    for (int w = w0; w < w1; ++w) nsc += hv.sc_cap[w];
    int kb = (nsc + 3) / 4;
    kb = kb < 1 ? 1 : (kb > hv.n_sm * 16 ? hv.n_sm * 16 : kb);
    const int a0 = hv.alch_base[w0], a1 = hv.alch_base[w1 - 1] + hv.n_alch[w1 - 1];
    k_quantize<<<sb, 256, 0, s>>>(d, g0, g1);
    k_colscan<<<nw, 32, 0, s>>>(d, w0);
    k_scatter<<<sb, 256, 0, s>>>(d, g0, g1);
    dim3 cg(max_cols < 1024 ? max_cols : 1024, nw);
    k_colsort<<<cg, 256, 0, s>>>(d, w0);
    k_kdsplit<<<kb, 128, 0, s>>>(d, w0, w1);
    k_permute_gather<<<sb, 256, 0, s>>>(d, g0, g1);
    k_permute_scatter<<<sb, 256, 0, s>>>(d, g0, g1);
    {
        long long nlb = ((long long)nsc * hv.ncs + LB_WARPS - 1) / LB_WARPS;
        int lb = (int)(nlb < (long long)hv.n_sm * 8 ? nlb : (long long)hv.n_sm * 8);  // resident grid
        k_listbuild<<<lb < 1 ? 1 : lb, LB_WARPS * 32, 0, s>>>(d, w0, w1);
        k_listcompact<<<kb, 128, 0, s>>>(d, w0, w1);
    }
    if (a1 > a0) {
        int ab = a1 - a0;
        ab = ab > hv.n_sm * 8 ? hv.n_sm * 8 : ab;
        k_alchlist<<<ab, AL_WARPS * 32, 0, s>>>(d, w0, w1, a0, a1);
    }
    k_items<<<nw, 256, 0, s>>>(d, w0, batched ? 1 : 0);
}

void launch_items(const Dev &d, const HostView &, int w0, int w1, cudaStream_t s) {
    k_items<<<w1 - w0, 256, 0, s>>>(d, w0, 0);
}

int rebuild_kernel_count(const HostView &hv, int w0, int w1) {
    const int a0 = hv.alch_base[w0], a1 = hv.alch_base[w1 - 1] + hv.n_alch[w1 - 1];
    return a1 > a0 ? 11 : 10;
}

}  // namespace labf
