// labf_api.cu -- host engine behind the C ABI of include/labf.h: layout of
// the device arena, upload of systems, the batched step as a CUDA graph, the
// one-walker-per-launch form, read-outs and the launch-shape autotuner.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "labf_internal.cuh"
#include "labf_launch.h"

using namespace labf;

namespace {

// an NVTX range over one C-ABI call (a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

constexpr size_t ALIGN = 256;
constexpr int IO_FLOATS_MIN = 1 << 16;

struct SysLayout {
    int n, n_alch, ncx, n_cols, sc_cap, slot_cap, W, P, Rq, cspan;
    double rho, r_list;
};

struct Layout {
    std::vector<SysLayout> sys;
    int W = 0, n_stages = 0, total_bins = 0, max_bins = 0, P_max = 1;
    long long slots = 0, scs = 0, cols = 0, atoms_w = 0, alch_w = 0, items = 0, bo = 0;
    long long atoms_s = 0, alch_s = 0, bonds = 0, angles = 0, posres = 0, fb = 0, lh = 0, lr = 0;
    int ent_cap = 0, alch_cap = 0, chunk = 32, max_n = 0, ncs = 1, sub_cap = 0;
    size_t bytes = 0;
};

struct Arena {
    char *base;
    size_t off, cap;
    bool dry;
    template <class T>
    T *take(size_t count) {
        off = (off + ALIGN - 1) / ALIGN * ALIGN;
        T *p = dry ? nullptr : reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

double steiner_box(double a, double b, double c, double r) {
    // volume of the box a x b x c dilated by a ball of radius r
    const double pi = 3.14159265358979323846;
    return a * b * c + 2.0 * (a * b + b * c + c * a) * r + pi * (a + b + c) * r * r +
           4.0 / 3.0 * pi * r * r * r;
}

int validate(const la_system_desc *sys, int n_sys, std::string &err) {
    if (!sys || n_sys <= 0) { err = "no systems"; return LA_ERR_INVALID_ARG; }
    int W = 0;
    for (int s = 0; s < n_sys; ++s) {
        const la_system_desc &S = sys[s];
        char buf[256];
        if (S.n_atoms <= 0 || !S.mass || !S.charge || !S.sigma || !S.epsilon || !S.alch ||
            !S.excl_group || !S.excl_extra || !S.x0 || !S.v0 || !S.lam0 || !S.plam0) {
            snprintf(buf, sizeof buf, "system %d: missing atom arrays or initial state", s);
            err = buf;
            return LA_ERR_INVALID_ARG;
        }
        if (!(S.box > 0) || !(S.r_cut > 0) || !(S.skin >= 0) || !(S.dt > 0) || !(S.kT > 0) ||
            !(S.m_lambda > 0) || S.n_stages <= 0 || S.n_stages > 16 || !S.stage_lo || !S.stage_hi ||
            !S.stage_bins || !S.stage_walkers || !(S.b_v > 0) || !(S.b_e < 1) || S.sc_n < 1 ||
            S.sc_m < 1 || !(S.n_full > 0) || S.shared_freq < 0) {
            snprintf(buf, sizeof buf, "system %d: invalid parameters", s);
            err = buf;
            return LA_ERR_INVALID_ARG;
        }
        if (S.box < 2.0 * (S.r_cut + S.skin)) {
            snprintf(buf, sizeof buf, "system %d: box %.4g < 2 (r_cut + skin) = %.4g", s, S.box,
                     2.0 * (S.r_cut + S.skin));
            err = buf;
            return LA_ERR_BOX_TOO_SMALL;
        }
        for (int k = 0; k < S.n_stages; ++k) {
            if (S.stage_bins[k] <= 0 || S.stage_walkers[k] < 1 || !(S.stage_hi[k] > S.stage_lo[k]) ||
                S.stage_lo[k] < 0.0 || S.stage_hi[k] > 1.0) {
                snprintf(buf, sizeof buf, "system %d: invalid stage %d", s, k);
                err = buf;
                return LA_ERR_INVALID_ARG;
            }
            W += S.stage_walkers[k];
        }
        for (int i = 0; i < S.n_atoms; ++i)
            if (!(S.mass[i] > 0)) {
                snprintf(buf, sizeof buf, "system %d: atom %d has non-positive mass", s, i);
                err = buf;
                return LA_ERR_INVALID_ARG;
            }
        auto chk = [&](int cnt, const int32_t *idx, int per) {
            if (cnt < 0) return false;
            if (cnt > 0 && !idx) return false;
            for (long long k = 0; k < (long long)cnt * per; ++k)
                if (idx[k] < 0 || idx[k] >= S.n_atoms) return false;
            return true;
        };
        if (!chk(S.n_bonds, S.bond_ij, 2) || !chk(S.n_angles, S.angle_ijk, 3) ||
            !chk(S.n_posres, S.posres_idx, 1) || !chk(S.n_fb_a, S.fb_a, 1) || !chk(S.n_fb_b, S.fb_b, 1) ||
            !chk(S.n_lh, S.lh_idx, 1) || !chk(S.n_lr, S.lr_ij, 2)) {
            snprintf(buf, sizeof buf, "system %d: topology index out of range", s);
            err = buf;
            return LA_ERR_INVALID_ARG;
        }
        if ((S.n_bonds && (!S.bond_r0 || !S.bond_k)) || (S.n_angles && (!S.angle_t0 || !S.angle_k)) ||
            (S.n_posres && !S.posres_x0) || (S.n_lh && !S.lh_x0)) {
            snprintf(buf, sizeof buf, "system %d: missing topology parameters", s);
            err = buf;
            return LA_ERR_INVALID_ARG;
        }
    }
    if (W <= 0 || W > LA_MAX_WALKERS_PER_LAUNCH) {
        err = "total walkers must be in [1, 256]";
        return LA_ERR_INVALID_ARG;
    }
    return LA_OK;
}

void compute_layout(const la_system_desc *sys, int n_sys, const la_options *opt, Layout &L) {
    const double fac = (opt && opt->list_capacity_factor >= 1.0) ? opt->list_capacity_factor : 1.6;
    L.chunk = (opt && opt->chunk_entries > 0) ? opt->chunk_entries : 32;
    const double pi = 3.14159265358979323846;
    double ent_est = 0.0, alch_est = 0.0, sub_est = 0.0;
    for (int s = 0; s < n_sys; ++s) {
        const la_system_desc &S = sys[s];
        SysLayout sl{};
        sl.n = S.n_atoms;
        sl.n_alch = 0;
        for (int i = 0; i < S.n_atoms; ++i) sl.n_alch += S.alch[i] ? 1 : 0;
        sl.P = 3 * sl.n_alch + 1;
        sl.rho = S.n_atoms / (S.box * S.box * S.box);
        sl.r_list = S.r_cut + S.skin;
        const double w_target = std::cbrt(64.0 / sl.rho);
        sl.ncx = std::max(1, std::min(255, (int)std::floor(S.box / w_target)));
        sl.n_cols = sl.ncx * sl.ncx;
        sl.sc_cap = (sl.n + SC - 1) / SC + sl.n_cols;
        sl.slot_cap = sl.sc_cap * SC;
        sl.W = 0;
        for (int k = 0; k < S.n_stages; ++k) sl.W += S.stage_walkers[k];
        const double wc = S.box / sl.ncx;
        const double h = std::min(S.box, 64.0 / (sl.rho * wc * wc));
        const double ej = std::cbrt(4.0 / sl.rho);
        // columns of the starting structures: the sparsest non-empty column
        // holds the tallest super-cluster (a lattice start can leave a column
        // with a thin sliver of atoms, whose one super-cluster spans the
        // whole box height), the densest one the most j-clusters in reach
        int cmin = 1 << 30, cmax = 0;
        {
            std::vector<int> cnt(sl.n_cols);
            const double binv = 1.0 / S.box;
            for (int w = 0; w < sl.W; ++w) {
                std::fill(cnt.begin(), cnt.end(), 0);
                for (int i = 0; i < S.n_atoms; ++i) {
                    int c2[2];
                    for (int q = 0; q < 2; ++q) {
                        const double t = (double)S.x0[3 * ((size_t)w * S.n_atoms + i) + q] * binv;
                        double f = (t - std::floor(t)) * 16777216.0;
                        unsigned long long u = (unsigned long long)std::floor(f);
                        if (u >= 16777216ull) u = 0;
                        c2[q] = (int)((u * (unsigned long long)sl.ncx) >> 24);
                    }
                    ++cnt[c2[0] + sl.ncx * c2[1]];
                }
                for (int c : cnt) {
                    if (c > 0) cmin = std::min(cmin, c);
                    cmax = std::max(cmax, c);
                }
            }
        }
        const double h_tall = cmax > 0 ? std::min(S.box, std::max(h, SC * S.box / (double)cmin)) : h;
        const double rho_dense = std::max(sl.rho, cmax / (wc * wc * S.box));
        const double V = steiner_box(wc + ej, wc + ej, h + ej, sl.r_list);
        const double V_tall = steiner_box(wc + ej, wc + ej, h_tall + ej, sl.r_list);
        const double full = std::min(std::max(sl.rho * V, rho_dense * V_tall) / JC, 27.0 * sl.sc_cap * NJC);
        ent_est = std::max(ent_est, full);
        // list radius in quantized units and the candidate columns per
        // dimension: a super-cluster box lies inside one column, so at most
        // floor(3 + 2 Rq ncx / 2^24) columns are within reach
        sl.Rq = (int)std::ceil(sl.r_list / S.box * 16777216.0) + 1;
        sl.cspan = (int)std::floor(3.0 + 2.0 * sl.Rq * (double)sl.ncx / 16777216.0);
        L.ncs = std::max(L.ncs, sl.cspan * sl.cspan);
        const double col_jc = std::max(sl.rho * wc * wc * (h + 2.0 * sl.r_list + 2.0 * ej),
                                       rho_dense * wc * wc * (h_tall + 2.0 * sl.r_list + 2.0 * ej)) / JC;
        const double col_cap = 3.0 * NJC * (std::max(sl.rho * wc * wc * S.box, (double)cmax) / SC + 2.0);
        sub_est = std::max(sub_est, std::min(col_jc, col_cap));
        alch_est = std::max(alch_est, sl.rho * 4.0 / 3.0 * pi * std::pow(sl.r_list, 3));
        L.sys.push_back(sl);
        L.W += sl.W;
        L.n_stages += S.n_stages;
        for (int k = 0; k < S.n_stages; ++k) {
            L.total_bins += S.stage_bins[k];
            L.max_bins = std::max(L.max_bins, S.stage_bins[k]);
        }
        L.P_max = std::max(L.P_max, sl.P);
        L.max_n = std::max(L.max_n, sl.n);
        L.slots += (long long)sl.W * sl.slot_cap;
        L.scs += (long long)sl.W * sl.sc_cap;
        L.cols += (long long)sl.W * sl.n_cols;
        L.atoms_w += (long long)sl.W * sl.n;
        L.alch_w += (long long)sl.W * sl.n_alch;
        L.bo += (long long)sl.W * (S.n_bonds + S.n_angles + S.n_posres);
        L.atoms_s += sl.n;
        L.alch_s += sl.n_alch;
        L.bonds += S.n_bonds;
        L.angles += S.n_angles;
        L.posres += S.n_posres;
        L.fb += S.n_fb_a + S.n_fb_b;
        L.lh += S.n_lh;
        L.lr += S.n_lr;
    }
    // the cyclic half list gives each super-cluster about half its neighbourhood
    L.ent_cap = (int)std::ceil(fac * 0.6 * ent_est) + 64;
    L.alch_cap = ((int)std::ceil(fac * alch_est) + 64 + 31) / 32 * 32;
    L.sub_cap = ((int)std::ceil(fac * sub_est) + 32 + 31) / 32 * 32;
    const int chunks = (L.ent_cap + L.chunk - 1) / L.chunk;
    L.items = L.scs * chunks;
}

// carve every device array out of the arena (dry run when base == nullptr)
// Arrays that carry the engine's state come first; the rebuild chain's and
// the list builder's scratch and the host I/O staging area come last, so that
// the state is the prefix [0, *state_bytes) (what a checkpoint copies).
size_t carve(const Layout &L, char *base, size_t cap, Dev &d, void **io, int *io_floats,
             SysDev **sysd, WalkerDev **walkd, StageDev **staged, size_t *state_bytes = nullptr) {
    Arena a{base, 0, cap, base == nullptr};
    *sysd = a.take<SysDev>(L.sys.size());
    *walkd = a.take<WalkerDev>(L.W);
    *staged = a.take<StageDev>(L.n_stages);
    d.ap = a.take<float4>(L.atoms_s);
    d.aparam_mut = a.take<float4>(L.atoms_s);
    d.anoise = a.take<float>(L.atoms_s);
    d.agroup = a.take<int>(L.atoms_s);
    d.aexcl = a.take<int4>(L.atoms_s);
    d.aalch = a.take<unsigned char>(L.atoms_s);
    d.alch_atoms = a.take<int>(std::max<long long>(1, L.alch_s));
    d.bond_ij = a.take<int2>(std::max<long long>(1, L.bonds));
    d.bond_p = a.take<float2>(std::max<long long>(1, L.bonds));
    d.angle_ijk = a.take<int4>(std::max<long long>(1, L.angles));
    d.angle_p = a.take<float2>(std::max<long long>(1, L.angles));
    d.posres_idx = a.take<int>(std::max<long long>(1, L.posres));
    d.posres_x0 = a.take<float4>(std::max<long long>(1, L.posres));
    d.fb_idx = a.take<int>(std::max<long long>(1, L.fb));
    d.lh_idx = a.take<int>(std::max<long long>(1, L.lh));
    d.lh_x0 = a.take<float4>(std::max<long long>(1, L.lh));
    d.lr_ij = a.take<int2>(std::max<long long>(1, L.lr));
    d.xq = a.take<float4>(L.slots);
    d.vv = a.take<float4>(L.slots);
    d.xref = a.take<float4>(L.slots);
    d.xprune = a.take<float4>(L.slots);
    d.lj = a.take<float2>(L.slots);
    d.im = a.take<float2>(L.slots);
    d.atom_of_slot = a.take<int>(L.slots);
    d.slot_walker = a.take<int>(L.slots);
    d.F = a.take<unsigned long long>(3 * L.slots);
    d.uq = a.take<int4>(L.slots);
    d.smeta = a.take<int2>(L.slots);
    d.sexcl = a.take<int4>(L.slots);
    d.slot_of_atom = a.take<int>(L.atoms_w);
    d.col_count = a.take<int>(L.cols);
    d.col_start = a.take<int>(L.cols);
    d.col_sc = a.take<int>(L.cols);
    d.col_nsc = a.take<int>(L.cols);
    d.n_sc = a.take<int>(L.W);
    d.sc_member = a.take<int>(L.scs * SC);
    d.sc_n = a.take<int>(L.scs);
    d.bb_sc = a.take<int4>(2 * L.scs);
    d.bb_ic = a.take<int4>(2 * L.scs * NIC);
    d.bb_jc = a.take<int4>(2 * L.scs * NJC);
    d.sc_nent = a.take<int>(L.scs);
    d.ent_hdr = a.take<int2>(L.scs * (long long)L.ent_cap);
    d.ent_lb = a.take<unsigned char>(32 * L.scs * (long long)L.ent_cap);
    d.items = a.take<int4>(L.items);
    d.n_items = a.take<int>(L.W);
    d.alch_cnt = a.take<int>(std::max<long long>(1, L.alch_w));
    d.alch_slot = a.take<int>(std::max<long long>(1, L.alch_w) * L.alch_cap);
    d.alch_out = a.take<double>(4 * std::max<long long>(1, L.alch_w));
    d.alch_th = a.take<double>(6 * std::max<long long>(1, L.alch_w));
    d.lam = a.take<double>(L.W);
    d.plam = a.take<double>(L.W);
    d.G = a.take<double>(L.W);
    d.s = a.take<double>(L.W);
    d.dl_direct = a.take<double>(L.W);
    d.wth = a.take<double>((size_t)L.W * 2 * L.P_max);
    d.step = a.take<unsigned long long>(L.W);
    d.pending = a.take<int>(L.W);
    d.rebuild = a.take<int>(L.W);
    d.prune = a.take<int>(L.W);
    d.near = a.take<int>(L.W);
    d.prune_now = a.take<unsigned long long>(L.W);
    d.eterm = a.take<long long>((size_t)L.W * N_ETERMS);
    d.abf_sum = a.take<double>(L.total_bins);
    d.abf_sumsq = a.take<double>(L.total_bins);
    d.abf_count = a.take<unsigned long long>(L.total_bins);
    d.dl_sum = a.take<double>((size_t)L.W * L.max_bins);
    d.dl_sumsq = a.take<double>((size_t)L.W * L.max_bins);
    d.dl_count = a.take<unsigned long long>((size_t)L.W * L.max_bins);
    d.th_d2 = a.take<double>((size_t)L.total_bins * L.P_max);
    d.th_d = a.take<double>((size_t)L.total_bins * L.P_max);
    d.th_sd = a.take<double>((size_t)L.total_bins * L.P_max);
    d.status = a.take<unsigned int>(4);
    d.counters = a.take<unsigned long long>(16);
    d.wdone = a.take<unsigned int>(L.W);
    d.sdone = a.take<unsigned int>(L.n_stages);
    if (state_bytes) *state_bytes = (a.off + ALIGN - 1) / ALIGN * ALIGN;
    // scratch: rewritten before every use
    d.t_xq = a.take<float4>(L.slots);
    d.t_vv = a.take<float4>(L.slots);
    d.t_old = a.take<int>(L.slots);
    d.t_uq = a.take<int4>(L.slots);
    d.t_col = a.take<int>(L.slots);
    d.t_pos = a.take<int>(L.slots);
    d.bucket = a.take<int>(L.atoms_w);
    d.sub_hdr = a.take<int2>(L.scs * (long long)L.ncs * L.sub_cap);
    d.sub_lb = a.take<unsigned char>(32 * L.scs * (long long)L.ncs * L.sub_cap);
    d.sub_n = a.take<int>(L.scs * (long long)L.ncs);
    const int iof = std::max(IO_FLOATS_MIN, 8 * L.max_n);
    *io = a.take<float>(iof);
    *io_floats = iof;
    return (a.off + ALIGN - 1) / ALIGN * ALIGN;
}

}  // namespace

struct la_handle {
    Layout L;
    Dev d{};
    HostView hv{};
    std::vector<SysDev> sys;
    std::vector<WalkerDev> walk;
    std::vector<StageDev> stages;
    std::vector<int> slot_off, slot_cap, sc_cap, n_cols, alch_base, n_alch, item_cap, bo_off, n_bo;
    std::vector<int> sys_w0;       // first walker of each system
    std::vector<int> sys_stage0;   // first stage of each system
    std::vector<int> sys_nstage;
    void *io = nullptr;
    int io_floats = 0;
    la_options opt{};
    int graph_steps = 10;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
    long long graph_launches_per_step = 0;
    int n_sm = 0, dev = 0;
    unsigned *h_status = nullptr;  // pinned
    cudaEvent_t status_ev = nullptr;
    int sticky = LA_OK;
    long long steps = 0, launches = 0, launches_per_step = 0;
    std::string err, report;
    bool dirty = false;  // a walker's state was set: lists and forces are refreshed lazily
    void *arena = nullptr;
    size_t state_bytes = 0;  // arena prefix holding the engine's state (checkpoints)
};

namespace {

int fail(la_handle *h, int code, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

#define CU(h, call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail(h, LA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int status_to_code(unsigned bits) {
    if (bits & (LA_STATUS_LIST_OVERFLOW | LA_STATUS_COLUMN_OVERFLOW | LA_STATUS_ALCH_OVERFLOW))
        return LA_ERR_LIST_OVERFLOW;
    if (bits & LA_STATUS_FIXED_OVERFLOW) return LA_ERR_FIXED_OVERFLOW;
    if (bits & LA_STATUS_NONFINITE) return LA_ERR_NONFINITE;
    if (bits & LA_STATUS_BAD_PARAM) return LA_ERR_INVALID_ARG;
    if (bits & LA_STATUS_BAD_INDEX) return LA_ERR_BAD_INDEX;
    return LA_OK;
}

const char *status_text(unsigned bits) {
    if (bits & LA_STATUS_COLUMN_OVERFLOW) return "a neighbour-search column exceeded 2048 atoms";
    if (bits & LA_STATUS_ALCH_OVERFLOW) return "an alchemical pair list exceeded its capacity";
    if (bits & LA_STATUS_LIST_OVERFLOW) return "the cluster-pair list exceeded its capacity";
    if (bits & LA_STATUS_FIXED_OVERFLOW) return "a force exceeded the fixed-point range";
    if (bits & LA_STATUS_NONFINITE) return "non-finite positions or lambda";
    if (bits & LA_STATUS_BAD_PARAM) return "negative or non-finite alchemical parameters";
    if (bits & LA_STATUS_BAD_INDEX) return "an index read from a device list was out of range (range-checked build)";
    return "ok";
}

// enqueue a copy of the status word to pinned memory after the call's work
void post_status(la_handle *h, cudaStream_t s) {
    cudaMemcpyAsync(h->h_status, h->d.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(h->status_ev, s);
}

int check_posted(la_handle *h) {
    if (h->sticky != LA_OK) return fail(h, LA_ERR_STATE, "handle in error state: %s", h->err.c_str());
    if (cudaEventQuery(h->status_ev) == cudaSuccess && *h->h_status) {
        int code = status_to_code(*h->h_status);
        if (code != LA_OK) {
            h->sticky = code;
            return fail(h, LA_ERR_STATE, "device error: %s", status_text(*h->h_status));
        }
    }
    return LA_OK;
}

int sync_status(la_handle *h, cudaStream_t s, unsigned *bits) {
    CU(h, cudaStreamSynchronize(s));
    unsigned st = 0;
    CU(h, cudaMemcpy(&st, h->d.status, sizeof st, cudaMemcpyDeviceToHost));
    if (bits) *bits = st;
    int code = status_to_code(st);
    if (code != LA_OK) {
        h->sticky = code;
        return fail(h, code, "device error: %s", status_text(st));
    }
    return LA_OK;
}

// one batched MD step over walkers [w0, w1)
// one batched MD step over all walkers: integrate, [rebuild], then one
// launch for pairs, bonded terms, walker terms and the lambda update
int enqueue_step(la_handle *h, int w0, int w1, cudaStream_t s) {
    launch_integrate(h->d, h->hv, w0, w1, s);
    launch_gate(h->d, w0, w1, 0, false, s);
    launch_rebuild(h->d, h->hv, w0, w1, s, true);
    launch_pairs_fused(h->d, h->hv, (int)h->stages.size(), s);
    return 0;
}

// integrate, gate, list kernels, fused pair launch
int kernels_per_step(la_handle *h) { return 1 + 1 + rebuild_kernel_count(h->hv, 0, h->L.W) + 1; }

// evaluate forces, dU/dlambda and G at the current state of walkers [w0, w1)
int prime(la_handle *h, int w0, int w1, bool force_rebuild, bool energy, cudaStream_t s) {
    if (force_rebuild) {
        std::vector<int> one(w1 - w0, 1);
        CU(h, cudaMemcpyAsync(h->d.rebuild + w0, one.data(), sizeof(int) * one.size(),
                              cudaMemcpyHostToDevice, s));
        CU(h, cudaStreamSynchronize(s));
    }
    const size_t g0 = h->slot_off[w0], g1 = (size_t)h->slot_off[w1 - 1] + h->slot_cap[w1 - 1];
    CU(h, cudaMemsetAsync(h->d.F + 3 * g0, 0, 3 * (g1 - g0) * sizeof(unsigned long long), s));
    if (energy) CU(h, cudaMemsetAsync(h->d.eterm + (size_t)N_ETERMS * w0, 0,
                                      sizeof(long long) * N_ETERMS * (w1 - w0), s));
    launch_rebuild(h->d, h->hv, w0, w1, s);
    launch_pairs(h->d, h->hv, w0, w1, energy, s);
    launch_bonded(h->d, h->hv, w0, w1, energy, s);
    launch_walker(h->d, w0, w1, energy, s);
    launch_lambda(h->d, 0, (int)h->stages.size(), true, s);
    h->launches += 4 + rebuild_kernel_count(h->hv, w0, w1);
    CU(h, cudaGetLastError());
    return LA_OK;
}

// lists and forces of walkers whose state la_set_state replaced (their
// rebuild flags are set), refreshed once for all before the next call
// that needs forces or lists
int flush_dirty(la_handle *h, cudaStream_t s) {
    if (!h->dirty) return LA_OK;
    h->dirty = false;
    return prime(h, 0, h->L.W, false, false, s);
}

int capture_graph(la_handle *h) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    // Each step: integrate -> gate -> IF(some walker must rebuild){rebuild
    // chain} -> pairs, bonded, walker, lambda.  The gate kernel sets the
    // step's conditional handle, so steps without a rebuild launch no list
    // kernel at all.
    const int W = h->L.W;
    h->launches_per_step = kernels_per_step(h);
    if (h->graph_steps == 0) return LA_OK;
    cudaStream_t cs = h->cap_stream, cb = h->cap_stream2;
    cudaGraph_t g;
    CU(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < h->graph_steps; ++k) {
        launch_integrate(h->d, h->hv, 0, W, cs);
        cudaStreamCaptureStatus st;
        cudaGraph_t cg;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        CU(h, cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle hc;
        CU(h, cudaGraphConditionalHandleCreate(&hc, cg, 0, cudaGraphCondAssignDefault));
        launch_gate(h->d, 0, W, hc, true, cs);
        CU(h, cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, &deps, nullptr, &nd));
        // IF (some walker must rebuild) { list kernels }
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = hc;
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        cudaGraphNode_t prev;
        CU(h, cudaGraphAddNode(&prev, cg, deps, nullptr, nd, &p));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        CU(h, cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        launch_rebuild(h->d, h->hv, 0, W, cb, true);
        cudaGraph_t body_out;
        CU(h, cudaStreamEndCapture(cb, &body_out));
        CU(h, cudaStreamUpdateCaptureDependencies(cs, &prev, nullptr, 1, cudaStreamSetCaptureDependencies));
        launch_pairs_fused(h->d, h->hv, (int)h->stages.size(), cs);
    }
    CU(h, cudaStreamEndCapture(cs, &g));
    cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, LA_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    // graph steps: integrate, gate, fused pairs; list kernels are counted per
    // step that runs them (device counter)
    h->graph_launches_per_step = h->launches_per_step - rebuild_kernel_count(h->hv, 0, W);
    return LA_OK;
}

void set_pair_blocks(la_handle *h, int ctas_per_sm) {
    h->hv.pair_blocks = std::max(1, ctas_per_sm) * h->n_sm;
}

// autotuner results per (device, system shape): CTAs/SM, entries/item, variant
std::mutex &tune_mutex() {  // handles may be created from several host threads
    static std::mutex m;
    return m;
}

std::map<std::string, std::array<int, 3>> &tune_cache() {
    static std::map<std::string, std::array<int, 3>> c;
    return c;
}

// forces, dU/dlambda and G of every walker from the current lists (no
// rebuild, no sample folded): bit-identical to what the last step left
int refresh_forces(la_handle *h, cudaStream_t s) {
    const int W = h->L.W;
    const size_t g1 = (size_t)h->slot_off[W - 1] + h->slot_cap[W - 1];
    CU(h, cudaMemsetAsync(h->d.F, 0, 3 * g1 * sizeof(unsigned long long), s));
    launch_pairs(h->d, h->hv, 0, W, false, s);
    launch_bonded(h->d, h->hv, 0, W, false, s);
    launch_walker(h->d, 0, W, false, s);
    launch_lambda(h->d, 0, (int)h->stages.size(), true, s);
    CU(h, cudaGetLastError());
    return LA_OK;
}

void make_report(la_handle *h) {
    static const char *vname[LA_PAIR_VARIANTS] = {"8 warps/CTA, 80 registers", "4 warps/CTA, 72 registers",
                                                  "4 warps/CTA, 64 registers"};
    char rep[512];
    snprintf(rep, sizeof rep,
             "%s: pair_variant=%d (%s), pair_ctas_per_sm=%d (8-warp CTA equivalents), "
             "chunk_entries=%d, graph steps=%d",
             h->opt.autotune ? "autotuned" : "fixed", h->hv.pair_variant, vname[h->hv.pair_variant],
             h->hv.pair_blocks / h->n_sm, h->d.chunk, h->graph_steps);
    h->report = rep;
}

// work items for the current chunk size from the current lists
int rebuild_items(la_handle *h, cudaStream_t s) {
    const int W = h->L.W;
    unsigned long long nreb = 0;
    CU(h, cudaMemcpyAsync(&nreb, h->d.counters, sizeof nreb, cudaMemcpyDeviceToHost, s));
    std::vector<int> one(W, 1);
    CU(h, cudaMemcpyAsync(h->d.rebuild, one.data(), sizeof(int) * W, cudaMemcpyHostToDevice, s));
    launch_items(h->d, h->hv, 0, W, s);
    CU(h, cudaMemcpyAsync(h->d.counters, &nreb, sizeof nreb, cudaMemcpyHostToDevice, s));  // not a rebuild
    CU(h, cudaStreamSynchronize(s));
    return LA_OK;
}

// Launch-shape tuner: times the pair kernel alone (repeated launches on the
// current lists, nothing else changes) for every variant, grid size and
// items size, keeps the fastest, then restores the forces exactly.
int tune_pairs(la_handle *h, cudaStream_t s, bool use_cache) {
    char key[256];
    snprintf(key, sizeof key, "dev%d-sm%d-W%d-slots%lld-ent%d", h->dev, h->n_sm, h->L.W, h->L.slots,
             h->L.ent_cap);
    int best_c = 4, best_k = h->L.chunk, best_m = 0;
    bool cached = false;
    if (use_cache) {
        std::lock_guard<std::mutex> lock(tune_mutex());
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            best_c = it->second[0];
            best_k = it->second[1];
            best_m = it->second[2];
            cached = true;
        }
    }
    if (!cached) {
        const int W = h->L.W;
        float best = 1e30f;
        const int ctas[] = {2, 3, 4, 6, 8};
        const int chunksz[] = {32, 64};  // item capacity was sized for L.chunk
        cudaEvent_t a, b;
        CU(h, cudaEventCreate(&a));
        CU(h, cudaEventCreate(&b));
        for (int k : chunksz) {
            if (k < h->L.chunk) continue;
            h->d.chunk = k;
            int rc = rebuild_items(h, s);
            if (rc != LA_OK) return rc;
            for (int m = 0; m < LA_PAIR_VARIANTS; ++m) {
                h->hv.pair_variant = m;
                for (int c : ctas) {
                    set_pair_blocks(h, c);
                    for (int r = 0; r < 2; ++r) launch_pairs(h->d, h->hv, 0, W, false, s);  // warm
                    CU(h, cudaEventRecord(a, s));
                    for (int r = 0; r < 10; ++r) launch_pairs(h->d, h->hv, 0, W, false, s);
                    CU(h, cudaEventRecord(b, s));
                    CU(h, cudaEventSynchronize(b));
                    float ms = 0.f;
                    CU(h, cudaEventElapsedTime(&ms, a, b));
                    if (ms < best) {
                        best = ms;
                        best_c = c;
                        best_k = k;
                        best_m = m;
                    }
                }
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        std::lock_guard<std::mutex> lock(tune_mutex());
        tune_cache()[key] = {best_c, best_k, best_m};
    }
    h->hv.pair_variant = best_m;
    set_pair_blocks(h, best_c);
    if (h->d.chunk != best_k) {
        h->d.chunk = best_k;
        int rc = rebuild_items(h, s);
        if (rc != LA_OK) return rc;
    }
    return refresh_forces(h, s);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int la_query_sizes(const la_system_desc *sys, int n_sys, const la_options *opt, size_t *arena_bytes) {
    std::string err;
    int rc = validate(sys, n_sys, err);
    if (rc != LA_OK) return rc;
    if (!arena_bytes) return LA_ERR_INVALID_ARG;
    Layout L;
    compute_layout(sys, n_sys, opt, L);
    Dev d{};
    void *io;
    int iof;
    SysDev *a;
    WalkerDev *b;
    StageDev *c;
    *arena_bytes = carve(L, nullptr, 0, d, &io, &iof, &a, &b, &c);
    return LA_OK;
}

int la_create_system(const la_system_desc *sys, int n_sys, const la_options *opt, void *arena,
                     size_t arena_bytes, void *stream, la_handle **out) {
    NvtxRange nvtx_range("la_create_system");
    if (!out) return LA_ERR_INVALID_ARG;
    *out = nullptr;
    la_handle *h = new la_handle();
    std::string err;
    int rc = validate(sys, n_sys, err);
    if (rc != LA_OK) {
        h->err = err;
        *out = h;
        return rc;
    }
    if (opt) h->opt = *opt;
    if (h->opt.pair_variant < 0 || h->opt.pair_variant >= LA_PAIR_VARIANTS ||
        (h->opt.chunk_entries > 0 && h->opt.chunk_entries % 32 != 0)) {
        h->err = "pair_variant must be in [0, LA_PAIR_VARIANTS) and chunk_entries a multiple of 32";
        *out = h;
        return LA_ERR_INVALID_ARG;
    }
    compute_layout(sys, n_sys, opt, h->L);
    const Layout &L = h->L;
    cudaStream_t s = (cudaStream_t)stream;
    SysDev *d_sys;
    WalkerDev *d_walk;
    StageDev *d_stage;
    size_t need = carve(L, (char *)arena, arena_bytes, h->d, &h->io, &h->io_floats, &d_sys, &d_walk, &d_stage,
                        &h->state_bytes);
    h->arena = arena;
    *out = h;
    if (!arena || need > arena_bytes || ((uintptr_t)arena % ALIGN) != 0)
        return fail(h, LA_ERR_ARENA_TOO_SMALL, "arena of %zu bytes (need %zu, 256-byte aligned)", arena_bytes, need);
    int dev;
    CU(h, cudaGetDevice(&dev));
    h->dev = dev;
    CU(h, cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));

    Dev &d = h->d;
    d.n_sys = n_sys;
    d.n_walkers = L.W;
    d.n_stages = L.n_stages;
    d.ent_cap = L.ent_cap;
    d.ncs = L.ncs;
    d.sub_cap = L.sub_cap;
    d.alch_cap = L.alch_cap;
    d.max_bins = L.max_bins;
    d.P_max = L.P_max;
    d.chunk = L.chunk;
    d.n_slots = (int)L.slots;
    d.n_scs = (int)L.scs;
    d.n_atoms_w = (int)L.atoms_w;
    d.n_atoms_s = (int)L.atoms_s;
    d.n_items_all = (int)L.items;
    d.sys = d_sys;
    d.walk = d_walk;
    d.stage = d_stage;

    // ---- per-system static data ----
    std::vector<float4> ap(L.atoms_s);
    std::vector<float> an(L.atoms_s);
    std::vector<int> ag(L.atoms_s), alch_atoms;
    std::vector<int4> ax(L.atoms_s);
    std::vector<unsigned char> aa(L.atoms_s);
    std::vector<int2> bij;
    std::vector<float2> bp, angp;
    std::vector<int4> aijk;
    std::vector<int> pidx, fbidx, lhidx;
    std::vector<int2> lrij;
    std::vector<float4> px0, lhx0;
    int atom_off = 0, alch_off = 0, stage_idx = 0, bin_off = 0;
    int w_glob = 0;
    long long slot_off = 0, sc_off = 0, col_off = 0, atom_base = 0, alch_base = 0, item_base = 0, bo = 0;
    const int chunks = (L.ent_cap + L.chunk - 1) / L.chunk;
    std::vector<float4> xq0(L.slots), vv0(L.slots);
    std::vector<float2> lj0(L.slots), im0(L.slots);
    std::vector<int> aos0(L.slots, -1), sw0(L.slots), soa0(L.atoms_w);
    std::vector<double> lam0(L.W), plam0(L.W);
    for (int si = 0; si < n_sys; ++si) {
        const la_system_desc &S = sys[si];
        const SysLayout &sl = L.sys[si];
        SysDev D{};
        D.n_atoms = S.n_atoms;
        D.atom_off = atom_off;
        D.n_alch = sl.n_alch;
        D.alch_off = alch_off;
        D.P = sl.P;
        D.box = S.box;
        D.box_inv = 1.0 / S.box;
        D.boxf = (float)S.box;
        D.box_invf = (float)(1.0 / S.box);
        D.rc2 = (float)(S.r_cut * S.r_cut);
        const double rc = S.r_cut;
        const double krf = S.eps_rf <= 0.0 ? 1.0 / (2.0 * rc * rc * rc)
                                           : (S.eps_rf - 1.0) / ((2.0 * S.eps_rf + 1.0) * rc * rc * rc);
        D.krf = (float)krf;
        D.crf = (float)(1.0 / rc + krf * rc * rc);
        D.sqrt_coul = (float)std::sqrt(std::max(0.0, S.coul));
        D.b_v = S.b_v;
        D.b_e = S.b_e;
        D.sc_alpha = (float)S.sc_alpha;
        D.sc_n = S.sc_n;
        D.sc_m = S.sc_m;
        D.dt = (float)S.dt;
        const double c_at = std::exp(-S.gamma * S.dt);
        D.c_at = (float)c_at;
        D.s_at = (float)std::sqrt(std::max(0.0, 1.0 - c_at * c_at));
        D.dt_d = S.dt;
        D.m_lambda = S.m_lambda;
        D.c_lm = std::exp(-S.gamma_lambda * S.dt);
        D.sd_lm = std::sqrt(std::max(0.0, (1.0 - D.c_lm * D.c_lm) * S.m_lambda * S.kT));
        D.kT = S.kT;
        D.half_skin2 = (float)(0.25 * S.skin * S.skin);
        D.near_skin2 = (float)(0.25 * S.skin * S.skin * NEAR_FRACTION * NEAR_FRACTION);
        {
            const double pm = h->opt.prune_margin;
            const bool on = pm > 0.0 && pm < S.skin;
            // a pruned tile holds no listed pair within r_c + pm; pruning is redone
            // once an atom moved 0.45 pm, so every pair moves less than 0.9 pm in
            // between (the 0.1 pm left covers FP32 rounding near the cutoff)
            D.prune_disp2 = on ? (float)(0.2025 * pm * pm) : 0.f;
            D.rprune2 = on ? (float)((S.r_cut + pm) * (S.r_cut + pm)) : 0.f;
        }
        const double binv = 1.0 / S.box;
        const double a_ = sl.r_list * binv;
        D.R = (long long)std::floor((a_ * a_) * 281474976710656.0);
        D.Rq = sl.Rq;
        D.ncx = sl.ncx;
        D.cspan = sl.cspan;
        D.bond_off = (int)bij.size();
        D.n_bonds = S.n_bonds;
        for (int b = 0; b < S.n_bonds; ++b) {
            bij.push_back(make_int2(S.bond_ij[2 * b], S.bond_ij[2 * b + 1]));
            bp.push_back(make_float2((float)S.bond_r0[b], (float)S.bond_k[b]));
        }
        D.angle_off = (int)aijk.size();
        D.n_angles = S.n_angles;
        for (int b = 0; b < S.n_angles; ++b) {
            aijk.push_back(make_int4(S.angle_ijk[3 * b], S.angle_ijk[3 * b + 1], S.angle_ijk[3 * b + 2], 0));
            angp.push_back(make_float2((float)S.angle_t0[b], (float)S.angle_k[b]));
        }
        D.posres_off = (int)pidx.size();
        D.n_posres = S.n_posres;
        D.posres_k = (float)S.posres_k;
        for (int b = 0; b < S.n_posres; ++b) {
            pidx.push_back(S.posres_idx[b]);
            px0.push_back(make_float4((float)S.posres_x0[3 * b], (float)S.posres_x0[3 * b + 1],
                                      (float)S.posres_x0[3 * b + 2], 0.f));
        }
        D.fb_off = (int)fbidx.size();
        D.n_fb_a = S.n_fb_a;
        D.n_fb_b = S.n_fb_b;
        D.fb_d0 = (float)S.fb_d0;
        D.fb_k = (float)S.fb_k;
        for (int b = 0; b < S.n_fb_a; ++b) fbidx.push_back(S.fb_a[b]);
        for (int b = 0; b < S.n_fb_b; ++b) fbidx.push_back(S.fb_b[b]);
        D.lh_off = (int)lhidx.size();
        D.n_lh = S.n_lh;
        D.lh_dims = S.lh_dims;
        D.lh_k0 = S.lh_k0;
        D.lh_k1 = S.lh_k1;
        D.lr_off = (int)lrij.size();
        D.n_lr = S.n_lr;
        D.lr_delta = S.lr_delta;
        D.lr_k = S.lr_k;
        for (int b = 0; b < S.n_lr; ++b) lrij.push_back(make_int2(S.lr_ij[2 * b], S.lr_ij[2 * b + 1]));
        for (int b = 0; b < S.n_lh; ++b) {
            lhidx.push_back(S.lh_idx[b]);
            lhx0.push_back(make_float4((float)S.lh_x0[3 * b], (float)S.lh_x0[3 * b + 1],
                                       (float)S.lh_x0[3 * b + 2], 0.f));
        }
        D.seed = S.seed;
        D.lambda_dynamics = S.lambda_dynamics;
        D.abf_on = S.abf_on;
        D.theta_stats = S.theta_stats;
        D.shared_freq = S.shared_freq > 0 ? S.shared_freq : 0;  // 0: host-managed merging
        D.n_full = S.n_full;
        D.w_first = w_glob;
        D.w_count = sl.W;
        h->sys.push_back(D);
        const double sqc = std::sqrt(std::max(0.0, S.coul));
        for (int i = 0; i < S.n_atoms; ++i) {
            ap[atom_off + i] = make_float4((float)(S.charge[i] * sqc), (float)(0.5 * S.sigma[i]),
                                           (float)(2.0 * std::sqrt(std::max(0.0, S.epsilon[i]))),
                                           (float)(1.0 / S.mass[i]));
            an[atom_off + i] = (float)std::sqrt(S.kT / S.mass[i]);
            ag[atom_off + i] = S.excl_group[i];
            ax[atom_off + i] = make_int4(S.excl_extra[4 * i], S.excl_extra[4 * i + 1], S.excl_extra[4 * i + 2],
                                         S.excl_extra[4 * i + 3]);
            aa[atom_off + i] = S.alch[i] ? 1 : 0;
            if (S.alch[i]) alch_atoms.push_back(i);
        }
        // stages and walkers
        h->sys_w0.push_back(w_glob);
        h->sys_stage0.push_back(stage_idx);
        h->sys_nstage.push_back(S.n_stages);
        int wl = 0;
        for (int k = 0; k < S.n_stages; ++k) {
            StageDev st{};
            st.sys = si;
            st.w0 = w_glob;
            st.w1 = w_glob + S.stage_walkers[k];
            st.n_bins = S.stage_bins[k];
            st.bin_off = bin_off;
            st.lo = S.stage_lo[k];
            st.hi = S.stage_hi[k];
            st.width = (st.hi - st.lo) / st.n_bins;
            bin_off += st.n_bins;
            for (int q = 0; q < S.stage_walkers[k]; ++q) {
                WalkerDev W{};
                W.sys = si;
                W.stage = stage_idx;
                W.wlocal = wl;
                W.slot_off = (int)slot_off;
                W.sc_cap = sl.sc_cap;
                W.sc_off = (int)sc_off;
                W.col_off = (int)col_off;
                W.n_cols = sl.n_cols;
                W.atom_base = (int)atom_base;
                W.alch_base = (int)alch_base;
                W.item_base = (int)item_base;
                W.item_cap = sl.sc_cap * chunks;
                W.bo_off = (int)bo;
                W.n_bo = S.n_bonds + S.n_angles + S.n_posres;
                // initial layout: slot = atom index, padding beyond
                const float *x = S.x0 + (size_t)wl * S.n_atoms * 3;
                const float *v = S.v0 + (size_t)wl * S.n_atoms * 3;
                for (int i = 0; i < sl.slot_cap; ++i) {
                    const size_t g = slot_off + i;
                    sw0[g] = w_glob;
                    if (i < S.n_atoms) {
                        xq0[g] = make_float4(x[3 * i], x[3 * i + 1], x[3 * i + 2], ap[atom_off + i].x);
                        vv0[g] = make_float4(v[3 * i], v[3 * i + 1], v[3 * i + 2], 0.f);
                        lj0[g] = make_float2(ap[atom_off + i].y, ap[atom_off + i].z);
                        im0[g] = make_float2(ap[atom_off + i].w, an[atom_off + i]);
                        aos0[g] = i;
                        soa0[atom_base + i] = (int)g;
                    } else {
                        xq0[g] = make_float4(x[0], x[1], x[2], 0.f);
                    }
                }
                lam0[w_glob] = S.lam0[wl];
                plam0[w_glob] = S.plam0[wl];
                h->walk.push_back(W);
                h->slot_off.push_back(W.slot_off);
                h->slot_cap.push_back(sl.slot_cap);
                h->sc_cap.push_back(sl.sc_cap);
                h->n_cols.push_back(sl.n_cols);
                h->alch_base.push_back(W.alch_base);
                h->n_alch.push_back(sl.n_alch);
                h->item_cap.push_back(W.item_cap);
                h->bo_off.push_back(W.bo_off);
                h->n_bo.push_back(W.n_bo);
                slot_off += sl.slot_cap;
                sc_off += sl.sc_cap;
                col_off += sl.n_cols;
                atom_base += sl.n;
                alch_base += sl.n_alch;
                item_base += W.item_cap;
                bo += W.n_bo;
                ++w_glob;
                ++wl;
            }
            h->stages.push_back(st);
            ++stage_idx;
        }
        atom_off += S.n_atoms;
        alch_off += sl.n_alch;
    }
    d.total_bo = (int)bo;
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        if (!bytes) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    // (re)load the whole initial state; also used to undo the autotuner's steps
    auto upload = [&]() -> int {
    CU(h, cudaMemsetAsync(arena, 0, need, s));
    CU(h, up(d_sys, h->sys.data(), sizeof(SysDev) * h->sys.size()));
    CU(h, up(d_walk, h->walk.data(), sizeof(WalkerDev) * h->walk.size()));
    CU(h, up(d_stage, h->stages.data(), sizeof(StageDev) * h->stages.size()));
    CU(h, up((void *)d.ap, ap.data(), sizeof(float4) * ap.size()));
    CU(h, up((void *)d.aparam_mut, ap.data(), sizeof(float4) * ap.size()));
    CU(h, up((void *)d.anoise, an.data(), sizeof(float) * an.size()));
    CU(h, up((void *)d.agroup, ag.data(), sizeof(int) * ag.size()));
    CU(h, up((void *)d.aexcl, ax.data(), sizeof(int4) * ax.size()));
    CU(h, up((void *)d.aalch, aa.data(), aa.size()));
    CU(h, up((void *)d.alch_atoms, alch_atoms.data(), sizeof(int) * alch_atoms.size()));
    CU(h, up((void *)d.bond_ij, bij.data(), sizeof(int2) * bij.size()));
    CU(h, up((void *)d.bond_p, bp.data(), sizeof(float2) * bp.size()));
    CU(h, up((void *)d.angle_ijk, aijk.data(), sizeof(int4) * aijk.size()));
    CU(h, up((void *)d.angle_p, angp.data(), sizeof(float2) * angp.size()));
    CU(h, up((void *)d.posres_idx, pidx.data(), sizeof(int) * pidx.size()));
    CU(h, up((void *)d.posres_x0, px0.data(), sizeof(float4) * px0.size()));
    CU(h, up((void *)d.fb_idx, fbidx.data(), sizeof(int) * fbidx.size()));
    CU(h, up((void *)d.lh_idx, lhidx.data(), sizeof(int) * lhidx.size()));
    CU(h, up((void *)d.lh_x0, lhx0.data(), sizeof(float4) * lhx0.size()));
    CU(h, up((void *)d.lr_ij, lrij.data(), sizeof(int2) * lrij.size()));
    CU(h, up(d.xq, xq0.data(), sizeof(float4) * xq0.size()));
    CU(h, up(d.vv, vv0.data(), sizeof(float4) * vv0.size()));
    CU(h, up(d.xref, xq0.data(), sizeof(float4) * xq0.size()));
    CU(h, up(d.lj, lj0.data(), sizeof(float2) * lj0.size()));
    CU(h, up(d.im, im0.data(), sizeof(float2) * im0.size()));
    CU(h, up(d.atom_of_slot, aos0.data(), sizeof(int) * aos0.size()));
    CU(h, up(d.slot_walker, sw0.data(), sizeof(int) * sw0.size()));
    CU(h, up(d.slot_of_atom, soa0.data(), sizeof(int) * soa0.size()));
    CU(h, up(d.lam, lam0.data(), sizeof(double) * lam0.size()));
    CU(h, up(d.plam, plam0.data(), sizeof(double) * plam0.size()));
    CU(h, cudaStreamSynchronize(s));
    return LA_OK;
    };
    rc = upload();
    if (rc != LA_OK) return rc;

    HostView &hv = h->hv;
    hv.n_walkers = L.W;
    hv.n_sm = h->n_sm;
    hv.ncs = L.ncs;
    hv.slot_off = h->slot_off.data();
    hv.slot_cap = h->slot_cap.data();
    hv.sc_cap = h->sc_cap.data();
    hv.n_cols = h->n_cols.data();
    hv.alch_base = h->alch_base.data();
    hv.n_alch = h->n_alch.data();
    hv.item_cap = h->item_cap.data();
    hv.bo_off = h->bo_off.data();
    hv.n_bo = h->n_bo.data();
    set_pair_blocks(h, h->opt.pair_ctas_per_sm > 0 ? h->opt.pair_ctas_per_sm : 4);
    h->hv.pair_variant = h->opt.pair_variant;
    // graph_steps < 0: no graph (one batched launch sequence per step)
    h->graph_steps = h->opt.graph_steps > 0 ? h->opt.graph_steps : (h->opt.graph_steps < 0 ? 0 : 10);

    CU(h, cudaMallocHost((void **)&h->h_status, sizeof(unsigned)));
    *h->h_status = 0;
    CU(h, cudaEventCreateWithFlags(&h->status_ev, cudaEventDisableTiming));
    CU(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CU(h, cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));

    rc = prime(h, 0, L.W, true, false, s);
    if (rc != LA_OK) return rc;
    rc = sync_status(h, s, nullptr);
    if (rc != LA_OK) return rc;

    // ---- launch-shape autotuner (pair kernel only; the state does not move) ----
    if (h->opt.autotune) {
        rc = tune_pairs(h, s, true);
        if (rc != LA_OK) return rc;
        rc = sync_status(h, s, nullptr);
        if (rc != LA_OK) return rc;
    }
    make_report(h);
    rc = capture_graph(h);
    if (rc != LA_OK) return rc;
    return sync_status(h, s, nullptr);
}

int la_step_walkers(la_handle *h, int64_t n_steps, void *stream) {
    NvtxRange nvtx_range("la_step_walkers");
    if (!h) return LA_ERR_INVALID_ARG;
    if (n_steps < 0) return fail(h, LA_ERR_INVALID_ARG, "n_steps < 0");
    int rc = check_posted(h);
    if (rc != LA_OK) return rc;
    if (n_steps == 0) return LA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    rc = flush_dirty(h, s);
    if (rc != LA_OK) return rc;
    const int64_t gs = h->graph_steps;
    const int64_t reps = gs > 0 ? n_steps / gs : 0, rem = gs > 0 ? n_steps % gs : n_steps;
    for (int64_t r = 0; r < reps; ++r) CU(h, cudaGraphLaunch(h->graph, s));
    for (int64_t r = 0; r < rem; ++r) enqueue_step(h, 0, h->L.W, s);
    launch_finish(h->d, h->hv, 0, h->L.W, s);
    CU(h, cudaGetLastError());
    h->steps += n_steps;
    h->launches += reps * h->graph_steps * h->graph_launches_per_step + rem * h->launches_per_step + 1;
    post_status(h, s);
    return LA_OK;
}

int la_step_walkers_plain(la_handle *h, int64_t n_steps, void *stream) {
    NvtxRange nvtx_range("la_step_walkers_plain");
    if (!h) return LA_ERR_INVALID_ARG;
    if (n_steps < 0) return fail(h, LA_ERR_INVALID_ARG, "n_steps < 0");
    int rc = check_posted(h);
    if (rc != LA_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = flush_dirty(h, s);
    if (rc != LA_OK) return rc;
    const int W = h->L.W;
    for (int64_t k = 0; k < n_steps; ++k) {
        // every walker's integrator runs before any rebuild: a walker that
        // moves too far flags all walkers of its system for this step
        for (int w = 0; w < W; ++w) launch_integrate(h->d, h->hv, w, w + 1, s);
        launch_coalesce(h->d, 0, W, s);  // the batched step's gate does the same
        h->launches += 1;
        for (int w = 0; w < W; ++w) {
            launch_rebuild(h->d, h->hv, w, w + 1, s);
            launch_pairs(h->d, h->hv, w, w + 1, false, s);
            launch_bonded(h->d, h->hv, w, w + 1, false, s);
            launch_walker(h->d, w, w + 1, false, s);
            h->launches += 3 + rebuild_kernel_count(h->hv, w, w + 1) + (h->n_bo[w] > 0 ? 1 : 0);
        }
        launch_lambda(h->d, 0, (int)h->stages.size(), false, s);
        h->launches += 1;
    }
    if (n_steps > 0) {
        for (int w = 0; w < W; ++w) launch_finish(h->d, h->hv, w, w + 1, s);
        h->launches += W;
    }
    CU(h, cudaGetLastError());
    h->steps += n_steps;
    post_status(h, s);
    return LA_OK;
}

int la_read_abf(la_handle *h, int sys, int stage, double *sum, double *sumsq, int64_t *count, double *grad,
                double *A, double *dA, double *dA_se, void *stream) {
    NvtxRange nvtx_range("la_read_abf");
    if (!h) return LA_ERR_INVALID_ARG;
    if (sys < 0 || sys >= (int)h->sys.size() || stage < 0 || stage >= h->sys_nstage[sys])
        return fail(h, LA_ERR_INVALID_ARG, "bad system/stage");
    cudaStream_t s = (cudaStream_t)stream;
    const StageDev &st = h->stages[h->sys_stage0[sys] + stage];
    const int nb = st.n_bins;
    std::vector<double> s1(nb), s2(nb);
    std::vector<unsigned long long> c(nb);
    CU(h, cudaMemcpyAsync(s1.data(), h->d.abf_sum + st.bin_off, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(s2.data(), h->d.abf_sumsq + st.bin_off, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(c.data(), h->d.abf_count + st.bin_off, sizeof(unsigned long long) * nb,
                          cudaMemcpyDeviceToHost, s));
    int rc = sync_status(h, s, nullptr);
    if (rc != LA_OK) return rc;
    // TI read-out (Sec. 2.3): Riemann sum of bin means
    const double w = st.width;
    double acc = 0.0, var_acc = 0.0;
    bool empty = false;
    if (A) A[0] = 0.0;
    for (int k = 0; k < nb; ++k) {
        if (sum) sum[k] = s1[k];
        if (sumsq) sumsq[k] = s2[k];
        if (count) count[k] = (int64_t)c[k];
        double g = std::nan("");
        if (c[k] > 0) {
            g = s1[k] / (double)c[k];
            const double var = std::max(0.0, s2[k] / (double)c[k] - g * g);
            var_acc += var / (double)c[k];
        } else {
            empty = true;
        }
        if (grad) grad[k] = g;
        acc += w * g;
        if (A) A[k + 1] = acc;
    }
    if (dA) *dA = acc;
    if (dA_se) *dA_se = empty ? std::nan("") : w * std::sqrt(var_acc);
    return empty ? LA_WARN_EMPTY_BIN : LA_OK;
}

int la_energy_forces(la_handle *h, int walker, uint32_t flags, double *energy_terms, float *forces, double *dUdl,
                     double *dUdtheta, double *d2Udl_dtheta, void *stream) {
    NvtxRange nvtx_range("la_energy_forces");
    if (!h) return LA_ERR_INVALID_ARG;
    if (walker < 0 || walker >= h->L.W) return fail(h, LA_ERR_INVALID_ARG, "bad walker");
    if (h->sticky != LA_OK) return fail(h, LA_ERR_STATE, "handle in error state: %s", h->err.c_str());
    cudaStream_t s = (cudaStream_t)stream;
    int rc = flush_dirty(h, s);
    if (rc != LA_OK) return rc;
    if (flags & LA_EF_COUNT_PAIRS) CU(h, cudaMemsetAsync(h->d.counters + 1, 0, 2 * sizeof(unsigned long long), s));
    rc = prime(h, walker, walker + 1, (flags & LA_EF_REBUILD) != 0, true, s);
    if (rc != LA_OK) return rc;
    const WalkerDev &W = h->walk[walker];
    const SysDev &S = h->sys[W.sys];
    if (forces) launch_forces_out(h->d, walker, S.n_atoms, forces, s);
    long long et[N_ETERMS];
    double sw = 0.0;
    std::vector<double> th(2 * h->L.P_max);
    CU(h, cudaMemcpyAsync(et, h->d.eterm + (size_t)N_ETERMS * walker, sizeof et, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(&sw, h->d.s + walker, sizeof sw, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(th.data(), h->d.wth + (size_t)walker * 2 * h->L.P_max, sizeof(double) * th.size(),
                          cudaMemcpyDeviceToHost, s));
    rc = sync_status(h, s, nullptr);
    if (rc != LA_OK) return rc;
    if (energy_terms)
        for (int k = 0; k < LA_N_TERMS; ++k) energy_terms[k] = (double)et[k] / E_TO_FIX;
    if (dUdl) *dUdl = sw;
    for (int p = 0; p < S.P; ++p) {
        if (dUdtheta) dUdtheta[p] = th[p];
        if (d2Udl_dtheta) d2Udl_dtheta[p] = th[h->L.P_max + p];
    }
    return LA_OK;
}

int la_energy_forces_device(la_handle *h, int walker, const float *x, const double *theta, const double *lam,
                            double *out, float *forces, void *stream) {
    NvtxRange nvtx_range("la_energy_forces_device");
    if (!h) return LA_ERR_INVALID_ARG;
    if (walker < 0 || walker >= h->L.W) return fail(h, LA_ERR_INVALID_ARG, "bad walker");
    int rc = check_posted(h);
    if (rc != LA_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = flush_dirty(h, s);
    if (rc != LA_OK) return rc;
    const WalkerDev &W = h->walk[walker];
    const SysDev &S = h->sys[W.sys];
    if (theta) {
        launch_alch_params_in(h->d, W.sys, S.n_alch, theta, s);
        h->dirty = true;  // the system's other walkers refresh before their next use
    }
    if (x) launch_positions_in(h->d, walker, S.n_atoms, x, s);
    if (lam) CU(h, cudaMemcpyAsync(h->d.lam + walker, lam, sizeof(double), cudaMemcpyDeviceToDevice, s));
    rc = prime(h, walker, walker + 1, false, true, s);
    if (rc != LA_OK) return rc;
    if (forces) launch_forces_out(h->d, walker, S.n_atoms, forces, s);
    if (out) launch_ef_out(h->d, walker, S.P, out, s);
    CU(h, cudaGetLastError());
    post_status(h, s);
    return LA_OK;
}

int la_get_state(la_handle *h, int walker, float *x, float *v, double *lam, double *plam, uint64_t *step,
                 void *stream) {
    if (!h) return LA_ERR_INVALID_ARG;
    if (walker < 0 || walker >= h->L.W) return fail(h, LA_ERR_INVALID_ARG, "bad walker");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->sys[h->walk[walker].sys].n_atoms;
    float *io = (float *)h->io;
    launch_state_io(h->d, walker, n, io, io + 3 * (size_t)n, false, s);
    std::vector<float> buf(6 * (size_t)n);
    CU(h, cudaMemcpyAsync(buf.data(), io, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost, s));
    double l = 0, p = 0;
    unsigned long long st = 0;
    CU(h, cudaMemcpyAsync(&l, h->d.lam + walker, sizeof l, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(&p, h->d.plam + walker, sizeof p, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(&st, h->d.step + walker, sizeof st, cudaMemcpyDeviceToHost, s));
    CU(h, cudaStreamSynchronize(s));
    if (x) memcpy(x, buf.data(), sizeof(float) * 3 * n);
    if (v) memcpy(v, buf.data() + 3 * (size_t)n, sizeof(float) * 3 * n);
    if (lam) *lam = l;
    if (plam) *plam = p;
    if (step) *step = st;
    return LA_OK;
}

int la_set_state(la_handle *h, int walker, const float *x, const float *v, const double *lam, const double *plam,
                 const uint64_t *step, void *stream) {
    if (!h) return LA_ERR_INVALID_ARG;
    if (walker < 0 || walker >= h->L.W) return fail(h, LA_ERR_INVALID_ARG, "bad walker");
    if (h->sticky != LA_OK) return fail(h, LA_ERR_STATE, "handle in error state: %s", h->err.c_str());
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->sys[h->walk[walker].sys].n_atoms;
    float *io = (float *)h->io;
    // the walker's lists and forces are stale from here on, whatever follows
    static const int one = 1;
    h->dirty = true;
    int rc = [&]() -> int {
        CU(h, cudaMemcpyAsync(h->d.rebuild + walker, &one, sizeof(int), cudaMemcpyHostToDevice, s));
        if (x || v) {
            // read back the current state first when one of the two stays unchanged
            if (!x || !v) launch_state_io(h->d, walker, n, io, io + 3 * (size_t)n, false, s);
            if (x) CU(h, cudaMemcpyAsync(io, x, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
            if (v) CU(h, cudaMemcpyAsync(io + 3 * (size_t)n, v, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
            launch_state_io(h->d, walker, n, io, io + 3 * (size_t)n, true, s);
        }
        if (lam) CU(h, cudaMemcpyAsync(h->d.lam + walker, lam, sizeof(double), cudaMemcpyHostToDevice, s));
        if (plam) CU(h, cudaMemcpyAsync(h->d.plam + walker, plam, sizeof(double), cudaMemcpyHostToDevice, s));
        if (step) CU(h, cudaMemcpyAsync(h->d.step + walker, step, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        return LA_OK;
    }();
    if (rc != LA_OK) {  // the walker may hold part of the new state
        h->sticky = rc;
        return rc;
    }
    return sync_status(h, s, nullptr);
}

int la_get_states(la_handle *h, float *x, float *v, double *lam, double *plam, uint64_t *step, void *stream) {
    NvtxRange nvtx_range("la_get_states");
    if (!h) return LA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int W = h->L.W;
    float *io = (float *)h->io;
    size_t off = 0;  // float offset of walker w's block in x and v
    for (int w = 0; w < W; ++w) {
        const int n = h->sys[h->walk[w].sys].n_atoms;
        if (x || v) {
            // the staging area is reused walker after walker: stream order puts
            // each copy-out before the next walker's gather
            launch_state_io(h->d, w, n, io, io + 3 * (size_t)n, false, s);
            if (x) CU(h, cudaMemcpyAsync(x + off, io, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
            if (v) CU(h, cudaMemcpyAsync(v + off, io + 3 * (size_t)n, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
        }
        off += 3 * (size_t)n;
    }
    if (lam) CU(h, cudaMemcpyAsync(lam, h->d.lam, sizeof(double) * W, cudaMemcpyDeviceToHost, s));
    if (plam) CU(h, cudaMemcpyAsync(plam, h->d.plam, sizeof(double) * W, cudaMemcpyDeviceToHost, s));
    if (step) CU(h, cudaMemcpyAsync(step, h->d.step, sizeof(uint64_t) * W, cudaMemcpyDeviceToHost, s));
    CU(h, cudaStreamSynchronize(s));
    return LA_OK;
}

int la_set_states(la_handle *h, const float *x, const float *v, const double *lam, const double *plam,
                  const uint64_t *step, void *stream) {
    NvtxRange nvtx_range("la_set_states");
    if (!h) return LA_ERR_INVALID_ARG;
    if (h->sticky != LA_OK) return fail(h, LA_ERR_STATE, "handle in error state: %s", h->err.c_str());
    cudaStream_t s = (cudaStream_t)stream;
    const int W = h->L.W;
    float *io = (float *)h->io;
    std::vector<int> one(W, 1);
    // every walker's lists and forces are stale from here on, whatever follows
    h->dirty = true;
    int rc = [&]() -> int {
        CU(h, cudaMemcpyAsync(h->d.rebuild, one.data(), sizeof(int) * W, cudaMemcpyHostToDevice, s));
        size_t off = 0;
        for (int w = 0; w < W; ++w) {
            const int n = h->sys[h->walk[w].sys].n_atoms;
            if (x || v) {
                // read back the current state first when one of the two stays unchanged
                if (!x || !v) launch_state_io(h->d, w, n, io, io + 3 * (size_t)n, false, s);
                if (x) CU(h, cudaMemcpyAsync(io, x + off, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
                if (v)
                    CU(h, cudaMemcpyAsync(io + 3 * (size_t)n, v + off, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
                launch_state_io(h->d, w, n, io, io + 3 * (size_t)n, true, s);
            }
            off += 3 * (size_t)n;
        }
        if (lam) CU(h, cudaMemcpyAsync(h->d.lam, lam, sizeof(double) * W, cudaMemcpyHostToDevice, s));
        if (plam) CU(h, cudaMemcpyAsync(h->d.plam, plam, sizeof(double) * W, cudaMemcpyHostToDevice, s));
        if (step) CU(h, cudaMemcpyAsync(h->d.step, step, sizeof(uint64_t) * W, cudaMemcpyHostToDevice, s));
        return LA_OK;
    }();
    if (rc != LA_OK) {  // some walkers may hold part of the new state
        cudaStreamSynchronize(s);
        h->sticky = rc;
        return rc;
    }
    return sync_status(h, s, nullptr);  // also keeps `one` alive until the copy is done
}

// ---- checkpoints: the arena's state prefix plus a header ----
namespace {
struct CkptHeader {
    char magic[8];
    uint64_t state_bytes, fingerprint;
    int32_t chunk, version;
    int64_t steps, launches;
};
constexpr int CKPT_VERSION = 1;

uint64_t fnv1a(uint64_t hsh, const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) hsh = (hsh ^ b[i]) * 1099511628211ull;
    return hsh;
}

// the layout and the per-system / per-walker / per-stage parameters: two
// engines built from the same inputs and options have the same fingerprint
uint64_t fingerprint(const la_handle *h) {
    uint64_t f = 14695981039346656037ull;
    f = fnv1a(f, &h->state_bytes, sizeof h->state_bytes);
    f = fnv1a(f, h->sys.data(), sizeof(SysDev) * h->sys.size());
    f = fnv1a(f, h->walk.data(), sizeof(WalkerDev) * h->walk.size());
    f = fnv1a(f, h->stages.data(), sizeof(StageDev) * h->stages.size());
    return f;
}
}  // namespace

int la_checkpoint_save(la_handle *h, void *buf, size_t cap, size_t *bytes, void *stream) {
    NvtxRange nvtx_range("la_checkpoint_save");
    if (!h || !bytes) return LA_ERR_INVALID_ARG;
    const size_t need = sizeof(CkptHeader) + h->state_bytes;
    *bytes = need;
    if (!buf) return LA_OK;
    if (cap < need) return fail(h, LA_ERR_INVALID_ARG, "checkpoint buffer of %zu bytes (need %zu)", cap, need);
    if (h->sticky != LA_OK) return fail(h, LA_ERR_STATE, "handle in error state: %s", h->err.c_str());
    cudaStream_t s = (cudaStream_t)stream;
    int rc = flush_dirty(h, s);  // lists and forces consistent with a state set last
    if (rc != LA_OK) return rc;
    CkptHeader hd{};
    memcpy(hd.magic, "LABFCKPT", 8);
    hd.state_bytes = h->state_bytes;
    hd.fingerprint = fingerprint(h);
    hd.chunk = h->d.chunk;
    hd.version = CKPT_VERSION;
    hd.steps = h->steps;
    hd.launches = h->launches;
    memcpy(buf, &hd, sizeof hd);
    CU(h, cudaMemcpyAsync((char *)buf + sizeof hd, h->arena, h->state_bytes, cudaMemcpyDeviceToHost, s));
    return sync_status(h, s, nullptr);
}

int la_checkpoint_load(la_handle *h, const void *buf, size_t bytes, void *stream) {
    NvtxRange nvtx_range("la_checkpoint_load");
    if (!h || !buf) return LA_ERR_INVALID_ARG;
    CkptHeader hd;
    if (bytes < sizeof hd) return fail(h, LA_ERR_INVALID_ARG, "checkpoint too short");
    memcpy(&hd, buf, sizeof hd);
    if (memcmp(hd.magic, "LABFCKPT", 8) != 0 || hd.version != CKPT_VERSION)
        return fail(h, LA_ERR_INVALID_ARG, "not a checkpoint of this library version");
    if (hd.state_bytes != h->state_bytes || bytes < sizeof hd + hd.state_bytes || hd.fingerprint != fingerprint(h))
        return fail(h, LA_ERR_INVALID_ARG, "checkpoint of a different system, layout or parameter set");
    if (hd.chunk != h->d.chunk)
        return fail(h, LA_ERR_INVALID_ARG, "checkpoint taken with chunk_entries=%d, this engine uses %d", hd.chunk,
                    h->d.chunk);
    cudaStream_t s = (cudaStream_t)stream;
    CU(h, cudaStreamSynchronize(s));
    CU(h, cudaMemcpyAsync(h->arena, (const char *)buf + sizeof hd, h->state_bytes, cudaMemcpyHostToDevice, s));
    h->dirty = false;
    h->steps = hd.steps;
    h->launches = hd.launches;
    h->sticky = LA_OK;
    return sync_status(h, s, nullptr);
}

int la_set_alch_params(la_handle *h, int sys, const double *theta, void *stream) {
    NvtxRange nvtx_range("la_set_alch_params");
    if (!h || !theta) return LA_ERR_INVALID_ARG;
    if (sys < 0 || sys >= (int)h->sys.size()) return fail(h, LA_ERR_INVALID_ARG, "bad system");
    cudaStream_t s = (cudaStream_t)stream;
    const SysDev &S = h->sys[sys];
    std::vector<int> idx(S.n_alch);
    CU(h, cudaMemcpy(idx.data(), h->d.alch_atoms + S.alch_off, sizeof(int) * S.n_alch, cudaMemcpyDeviceToHost));
    std::vector<float4> ap(S.n_atoms);
    CU(h, cudaMemcpy(ap.data(), h->d.aparam_mut + S.atom_off, sizeof(float4) * S.n_atoms, cudaMemcpyDeviceToHost));
    for (int r = 0; r < S.n_alch; ++r) {
        const double eps = theta[3 * r], sig = theta[3 * r + 1], q = theta[3 * r + 2];
        if (!(eps >= 0) || !(sig >= 0)) return fail(h, LA_ERR_INVALID_ARG, "negative epsilon or sigma");
        float4 &p = ap[idx[r]];
        p.x = (float)(q * S.sqrt_coul);
        p.y = (float)(0.5 * sig);
        p.z = (float)(2.0 * std::sqrt(eps));
    }
    CU(h, cudaMemcpyAsync(h->d.aparam_mut + S.atom_off, ap.data(), sizeof(float4) * S.n_atoms,
                          cudaMemcpyHostToDevice, s));
    const int w0 = h->sys_w0[sys];
    int w1 = w0;
    while (w1 < h->L.W && h->walk[w1].sys == sys) ++w1;
    int rc = prime(h, w0, w1, true, false, s);
    if (rc != LA_OK) return rc;
    return sync_status(h, s, nullptr);
}

int la_abf_export(la_handle *h, int sys, int stage, double *sum, double *sumsq, int64_t *count, void *stream) {
    NvtxRange nvtx_range("la_abf_export");
    if (!h || !sum || !sumsq || !count) return LA_ERR_INVALID_ARG;
    if (sys < 0 || sys >= (int)h->sys.size() || stage < 0 || stage >= h->sys_nstage[sys])
        return fail(h, LA_ERR_INVALID_ARG, "bad system/stage");
    cudaStream_t s = (cudaStream_t)stream;
    const StageDev &st = h->stages[h->sys_stage0[sys] + stage];
    const int MB = h->L.max_bins, nw = st.w1 - st.w0;
    std::vector<double> a((size_t)nw * MB), b((size_t)nw * MB);
    std::vector<unsigned long long> c((size_t)nw * MB);
    CU(h, cudaMemcpyAsync(a.data(), h->d.dl_sum + (size_t)st.w0 * MB, sizeof(double) * a.size(), cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(b.data(), h->d.dl_sumsq + (size_t)st.w0 * MB, sizeof(double) * b.size(), cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(c.data(), h->d.dl_count + (size_t)st.w0 * MB, sizeof(unsigned long long) * c.size(),
                          cudaMemcpyDeviceToHost, s));
    int rc = sync_status(h, s, nullptr);
    if (rc != LA_OK) return rc;
    for (int k = 0; k < st.n_bins; ++k) {
        double s1 = 0.0, s2 = 0.0;
        unsigned long long n = 0;
        for (int w = 0; w < nw; ++w) {  // walker order
            s1 += a[(size_t)w * MB + k];
            s2 += b[(size_t)w * MB + k];
            n += c[(size_t)w * MB + k];
        }
        sum[k] = s1;
        sumsq[k] = s2;
        count[k] = (int64_t)n;
    }
    return LA_OK;
}

int la_abf_import(la_handle *h, int sys, int stage, const double *sum, const double *sumsq, const int64_t *count,
                  void *stream) {
    NvtxRange nvtx_range("la_abf_import");
    if (!h || !sum || !sumsq || !count) return LA_ERR_INVALID_ARG;
    if (sys < 0 || sys >= (int)h->sys.size() || stage < 0 || stage >= h->sys_nstage[sys])
        return fail(h, LA_ERR_INVALID_ARG, "bad system/stage");
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = flush_dirty(h, s);
    if (rc0 != LA_OK) return rc0;
    const StageDev &st = h->stages[h->sys_stage0[sys] + stage];
    const int nb = st.n_bins, MB = h->L.max_bins;
    std::vector<double> s1(nb), s2(nb);
    std::vector<unsigned long long> c(nb);
    CU(h, cudaMemcpyAsync(s1.data(), h->d.abf_sum + st.bin_off, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(s2.data(), h->d.abf_sumsq + st.bin_off, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(c.data(), h->d.abf_count + st.bin_off, sizeof(unsigned long long) * nb,
                          cudaMemcpyDeviceToHost, s));
    CU(h, cudaStreamSynchronize(s));
    for (int k = 0; k < nb; ++k) {
        if (count[k] < 0) return fail(h, LA_ERR_INVALID_ARG, "negative count");
        s1[k] += sum[k];
        s2[k] += sumsq[k];
        c[k] += (unsigned long long)count[k];
    }
    CU(h, cudaMemcpyAsync(h->d.abf_sum + st.bin_off, s1.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    CU(h, cudaMemcpyAsync(h->d.abf_sumsq + st.bin_off, s2.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    CU(h, cudaMemcpyAsync(h->d.abf_count + st.bin_off, c.data(), sizeof(unsigned long long) * nb,
                          cudaMemcpyHostToDevice, s));
    const size_t rows = (size_t)(st.w1 - st.w0) * MB;
    CU(h, cudaMemsetAsync(h->d.dl_sum + (size_t)st.w0 * MB, 0, sizeof(double) * rows, s));
    CU(h, cudaMemsetAsync(h->d.dl_sumsq + (size_t)st.w0 * MB, 0, sizeof(double) * rows, s));
    CU(h, cudaMemsetAsync(h->d.dl_count + (size_t)st.w0 * MB, 0, sizeof(unsigned long long) * rows, s));
    // refresh the lambda forces with the new bias
    launch_lambda(h->d, 0, (int)h->stages.size(), true, s);
    return sync_status(h, s, nullptr);
}

int la_read_theta(la_handle *h, int sys, int stage, double *sum_d2, double *sum_d, double *sum_sd,
                  double *dA_dtheta, void *stream) {
    NvtxRange nvtx_range("la_read_theta");
    if (!h) return LA_ERR_INVALID_ARG;
    if (sys < 0 || sys >= (int)h->sys.size() || stage < 0 || stage >= h->sys_nstage[sys])
        return fail(h, LA_ERR_INVALID_ARG, "bad system/stage");
    cudaStream_t s = (cudaStream_t)stream;
    const StageDev &st = h->stages[h->sys_stage0[sys] + stage];
    const int P = h->sys[sys].P, PM = h->L.P_max, nb = st.n_bins, MB = h->L.max_bins;
    std::vector<double> th[3];
    double *srcs[3] = {h->d.th_d2, h->d.th_d, h->d.th_sd};
    for (int q = 0; q < 3; ++q) {
        th[q].resize((size_t)nb * PM);
        CU(h, cudaMemcpyAsync(th[q].data(), srcs[q] + (size_t)st.bin_off * PM, sizeof(double) * th[q].size(),
                              cudaMemcpyDeviceToHost, s));
    }
    // samples per bin (merged and walker-local) and their dU/dlambda sums
    std::vector<double> s1(nb), l1((size_t)h->L.W * MB);
    std::vector<unsigned long long> c(nb), lc((size_t)h->L.W * MB);
    CU(h, cudaMemcpyAsync(s1.data(), h->d.abf_sum + st.bin_off, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(c.data(), h->d.abf_count + st.bin_off, sizeof(unsigned long long) * nb,
                          cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(l1.data(), h->d.dl_sum, sizeof(double) * l1.size(), cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(lc.data(), h->d.dl_count, sizeof(unsigned long long) * lc.size(), cudaMemcpyDeviceToHost, s));
    int rc = sync_status(h, s, nullptr);
    if (rc != LA_OK) return rc;
    double *outs[3] = {sum_d2, sum_d, sum_sd};
    for (int q = 0; q < 3; ++q)
        if (outs[q])
            for (int k = 0; k < nb; ++k)
                for (int p = 0; p < P; ++p) outs[q][(size_t)k * P + p] = th[q][(size_t)k * PM + p];
    if (dA_dtheta) {
        // d Delta A / d theta = sum_k w [<d2U/dl dth> - beta Cov(dU/dl, dU/dth)]
        // (the lambda-conditional ensemble depends on theta, hence the covariance)
        const double beta = 1.0 / h->sys[sys].kT;
        for (int p = 0; p < P; ++p) dA_dtheta[p] = 0.0;
        for (int k = 0; k < nb; ++k) {
            double sum = s1[k], cnt = (double)c[k];
            for (int w = st.w0; w < st.w1; ++w) {
                sum += l1[(size_t)w * MB + k];
                cnt += (double)lc[(size_t)w * MB + k];
            }
            if (cnt <= 0.0) {
                for (int p = 0; p < P; ++p) dA_dtheta[p] = std::nan("");
                rc = LA_WARN_EMPTY_BIN;
                continue;
            }
            const double ms = sum / cnt;
            for (int p = 0; p < P; ++p) {
                const double m2 = th[0][(size_t)k * PM + p] / cnt, md = th[1][(size_t)k * PM + p] / cnt;
                const double msd = th[2][(size_t)k * PM + p] / cnt;
                dA_dtheta[p] += st.width * (m2 - beta * (msd - ms * md));
            }
        }
    }
    return rc;
}

int la_get_pairs(la_handle *h, int walker, int32_t *pairs, uint8_t *kind, int64_t cap, int64_t *count,
                 void *stream) {
    NvtxRange nvtx_range("la_get_pairs");
    if (!h || !count) return LA_ERR_INVALID_ARG;
    if (walker < 0 || walker >= h->L.W) return fail(h, LA_ERR_INVALID_ARG, "bad walker");
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = flush_dirty(h, s);
    if (rc0 != LA_OK) return rc0;
    CU(h, cudaStreamSynchronize(s));
    const WalkerDev &W = h->walk[walker];
    const SysDev &S = h->sys[W.sys];
    const int nslot = h->slot_cap[walker];
    std::vector<int> aos(nslot), nent(W.sc_cap);
    int nsc = 0;
    CU(h, cudaMemcpy(aos.data(), h->d.atom_of_slot + W.slot_off, sizeof(int) * nslot, cudaMemcpyDeviceToHost));
    CU(h, cudaMemcpy(&nsc, h->d.n_sc + walker, sizeof(int), cudaMemcpyDeviceToHost));
    CU(h, cudaMemcpy(nent.data(), h->d.sc_nent + W.sc_off, sizeof(int) * W.sc_cap, cudaMemcpyDeviceToHost));
    std::vector<int2> hdr((size_t)W.sc_cap * h->L.ent_cap);
    std::vector<unsigned char> lbs(32 * hdr.size());
    CU(h, cudaMemcpy(hdr.data(), h->d.ent_hdr + (size_t)W.sc_off * h->L.ent_cap, sizeof(int2) * hdr.size(),
                     cudaMemcpyDeviceToHost));
    CU(h, cudaMemcpy(lbs.data(), h->d.ent_lb + 32 * (size_t)W.sc_off * h->L.ent_cap, lbs.size(),
                     cudaMemcpyDeviceToHost));
    std::vector<std::pair<long long, int>> out;
    for (int sl = 0; sl < nsc; ++sl) {
        for (int e = 0; e < nent[W.sc_off + sl - W.sc_off]; ++e) {
            const size_t ge = (size_t)sl * h->L.ent_cap + e;
            const int jbase = hdr[ge].x - W.slot_off;
            const unsigned imask = ((unsigned)hdr[ge].y >> 16) & 0xffu;  // listed, not pruned
            for (int ic = 0; ic < NIC; ++ic) {
                if (!(imask & (1u << ic))) continue;
                for (int lane = 0; lane < 32; ++lane) {
                    if (!(lbs[32 * ge + lane] & (1u << ic))) continue;
                    const int a = aos[sl * SC + ic * IC + (lane & 7)], b = aos[jbase + (lane >> 3)];
                    const int i = std::min(a, b), j = std::max(a, b);
                    out.push_back({(long long)i * S.n_atoms + j, 0});
                }
            }
        }
    }
    const int na = S.n_alch;
    if (na > 0) {
        std::vector<int> acnt(na), aslot((size_t)na * h->L.alch_cap), aidx(na);
        CU(h, cudaMemcpy(acnt.data(), h->d.alch_cnt + W.alch_base, sizeof(int) * na, cudaMemcpyDeviceToHost));
        CU(h, cudaMemcpy(aslot.data(), h->d.alch_slot + (size_t)W.alch_base * h->L.alch_cap,
                         sizeof(int) * aslot.size(), cudaMemcpyDeviceToHost));
        CU(h, cudaMemcpy(aidx.data(), h->d.alch_atoms + S.alch_off, sizeof(int) * na, cudaMemcpyDeviceToHost));
        for (int r = 0; r < na; ++r)
            for (int k = 0; k < acnt[r]; ++k) {
                const int b = aos[aslot[(size_t)r * h->L.alch_cap + k] - W.slot_off];
                const int a = aidx[r];
                out.push_back({(long long)std::min(a, b) * S.n_atoms + std::max(a, b), 1});
            }
    }
    std::sort(out.begin(), out.end());
    *count = (int64_t)out.size();
    for (size_t k = 0; k < out.size() && (int64_t)k < cap; ++k) {
        if (pairs) {
            pairs[2 * k] = (int32_t)(out[k].first / S.n_atoms);
            pairs[2 * k + 1] = (int32_t)(out[k].first % S.n_atoms);
        }
        if (kind) kind[k] = (uint8_t)out[k].second;
    }
    return LA_OK;
}

int la_lambda_path(la_handle *h, const double *lam, int n, double b_v, double b_e, double *out, void *stream) {
    if (!h || !lam || !out || n < 0) return LA_ERR_INVALID_ARG;
    if ((size_t)n * 5 * sizeof(double) > (size_t)h->io_floats * sizeof(float))
        return fail(h, LA_ERR_INVALID_ARG, "too many lambda values for the I/O buffer");
    if (n == 0) return LA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    double *dl = (double *)h->io, *dout = dl + n;
    CU(h, cudaMemcpyAsync(dl, lam, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    launch_lambda_path(dl, n, b_v, b_e, dout, s);
    CU(h, cudaMemcpyAsync(out, dout, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s));
    CU(h, cudaStreamSynchronize(s));
    return LA_OK;
}

int la_sync(la_handle *h, void *stream, uint32_t *status_bits) {
    if (!h) return LA_ERR_INVALID_ARG;
    unsigned bits = 0;
    int rc = sync_status(h, (cudaStream_t)stream, &bits);
    if (status_bits) *status_bits = bits;
    return rc;
}

int la_stats(la_handle *h, int64_t *out, void *stream) {
    if (!h) return LA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long c[12];
    CU(h, cudaMemcpyAsync(c, h->d.counters, sizeof c, cudaMemcpyDeviceToHost, s));
    std::vector<int> nent(h->L.scs), nsc(h->L.W);
    CU(h, cudaMemcpyAsync(nent.data(), h->d.sc_nent, sizeof(int) * nent.size(), cudaMemcpyDeviceToHost, s));
    CU(h, cudaMemcpyAsync(nsc.data(), h->d.n_sc, sizeof(int) * nsc.size(), cudaMemcpyDeviceToHost, s));
    CU(h, cudaStreamSynchronize(s));
    long long ents = 0, tiles = 0;
    std::vector<int2> hdr(h->L.ent_cap);
    for (int w = 0; w < h->L.W; ++w)
        for (int k = 0; k < nsc[w]; ++k) {
            const int sc = h->walk[w].sc_off + k;
            const int ne = nent[sc];
            ents += ne;
            if (ne <= 0) continue;
            CU(h, cudaMemcpy(hdr.data(), h->d.ent_hdr + (size_t)sc * h->L.ent_cap, sizeof(int2) * ne,
                             cudaMemcpyDeviceToHost));
            for (int e = 0; e < ne; ++e) tiles += __builtin_popcount(((unsigned)hdr[e].y >> 8) & 0xffu);
        }
    if (out) {
        out[0] = h->steps;
        out[1] = (int64_t)c[0];
        // list kernels run inside the graph only on rebuild steps (counted by the gate)
        out[2] = h->launches + (int64_t)c[6] * rebuild_kernel_count(h->hv, 0, h->L.W);
        out[3] = (int64_t)c[1];
        out[4] = (int64_t)c[2];
        out[5] = ents;
        out[6] = tiles;
        out[7] = (int64_t)c[10];
    }
    return LA_OK;
}

int la_time_kernels(la_handle *h, int n_steps, float *ms_out, int64_t *launches_out, void *stream) {
    NvtxRange nvtx_range("la_time_kernels");
    if (!h || !ms_out || n_steps <= 0) return LA_ERR_INVALID_ARG;
    int rc = check_posted(h);
    if (rc != LA_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = flush_dirty(h, s);
    if (rc != LA_OK) return rc;
    const int W = h->L.W;
    // integrate | gate | (host reads the flags) | list kernels when a walker
    // must rebuild | fused pair launch; the host's gap is in no class
    cudaEvent_t ev[6];
    for (auto &e : ev) CU(h, cudaEventCreate(&e));
    double acc[LA_N_KERNELS] = {0};
    int64_t cnt[LA_N_KERNELS] = {0};
    std::vector<int> flags(W);
    for (int k = 0; k < n_steps; ++k) {
        cudaEventRecord(ev[0], s);
        launch_integrate(h->d, h->hv, 0, W, s);
        cudaEventRecord(ev[1], s);
        launch_gate(h->d, 0, W, 0, false, s);
        cudaEventRecord(ev[2], s);
        // the graph's conditional node runs the list kernels only on steps
        // where some walker must rebuild: read the flags the integrator set
        CU(h, cudaMemcpyAsync(flags.data(), h->d.rebuild, sizeof(int) * W, cudaMemcpyDeviceToHost, s));
        CU(h, cudaStreamSynchronize(s));
        bool any = false;
        for (int w = 0; w < W; ++w) any = any || flags[w] != 0;
        cudaEventRecord(ev[3], s);
        if (any) launch_rebuild(h->d, h->hv, 0, W, s, true);
        cudaEventRecord(ev[4], s);
        // the fused launch of the batched step: pairs, bonded terms, walker
        // terms and the lambda update
        launch_pairs_fused(h->d, h->hv, (int)h->stages.size(), s);
        cudaEventRecord(ev[5], s);
        CU(h, cudaEventSynchronize(ev[5]));
        float t01 = 0.f, t12 = 0.f, t34 = 0.f, t45 = 0.f;
        cudaEventElapsedTime(&t01, ev[0], ev[1]);
        cudaEventElapsedTime(&t12, ev[1], ev[2]);
        cudaEventElapsedTime(&t34, ev[3], ev[4]);
        cudaEventElapsedTime(&t45, ev[4], ev[5]);
        acc[0] += t01;
        acc[1] += t12 + (any ? t34 : 0.f);
        acc[2] += t45;  // bonded, walker, lambda run inside the pair launch: 0
        cnt[0] += 1;
        cnt[1] += 1 + (any ? rebuild_kernel_count(h->hv, 0, W) : 0);
        cnt[2] += 1;
    }
    launch_finish(h->d, h->hv, 0, W, s);
    h->steps += n_steps;
    h->launches += cnt[0] + cnt[1] + cnt[2] + 1;
    for (auto &e : ev) cudaEventDestroy(e);
    for (int q = 0; q < LA_N_KERNELS; ++q) {
        ms_out[q] = (float)(acc[q] / n_steps);
        if (launches_out) launches_out[q] = cnt[q];
    }
    return sync_status(h, s, nullptr);
}

int la_autotune(la_handle *h, void *stream) {
    NvtxRange nvtx_range("la_autotune");
    if (!h) return LA_ERR_INVALID_ARG;
    int rc = check_posted(h);
    if (rc != LA_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = flush_dirty(h, s);
    if (rc != LA_OK) return rc;
    rc = sync_status(h, s, nullptr);
    if (rc != LA_OK) return rc;
    rc = tune_pairs(h, s, false);
    if (rc != LA_OK) return rc;
    h->opt.autotune = 1;
    make_report(h);
    rc = capture_graph(h);
    if (rc != LA_OK) return rc;
    return sync_status(h, s, nullptr);
}

const char *la_autotune_report(la_handle *h) { return h ? h->report.c_str() : "no handle"; }

const char *la_last_error(la_handle *h) { return h ? h->err.c_str() : "no handle"; }

int la_destroy(la_handle *h) {
    if (!h) return LA_OK;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
    if (h->status_ev) cudaEventDestroy(h->status_ev);
    if (h->h_status) cudaFreeHost(h->h_status);
    delete h;
    return LA_OK;
}

}  // extern "C"
