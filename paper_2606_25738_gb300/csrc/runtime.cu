// Host runtime of the row-wise PairHMM library: the C ABI of include/phmm.h, contexts,
// per-ticket device arenas, the work planner (length buckets and team packing), the
// built-in tuner for N, CUDA-graph capture and replay, and ticket polling.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <array>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "launch.h"
#include "phmm.h"
#include "phmm_internal.h"

using namespace phmm;

namespace {

// ------------------------------------------------------------------------------------
// Buffers
// ------------------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};
struct HostBuf {
    void* p = nullptr;
    size_t cap = 0;
};

cudaError_t ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return cudaSuccess;
    const bool regrow = b.cap > 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    // regrowth keeps 1/8 headroom so that batches of slowly varying size reallocate rarely
    // (cudaFree waits for the whole device, including other slots' work)
    const size_t nb = std::max(regrow ? bytes + bytes / 8 : bytes, (size_t)4096);
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.cap = nb;
    return cudaSuccess;
}
cudaError_t ensure(HostBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return cudaSuccess;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMallocHost(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.cap = bytes;
    return cudaSuccess;
}
void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}
void release(HostBuf& b) {
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
}

// ------------------------------------------------------------------------------------
// Work plan
// ------------------------------------------------------------------------------------
struct Plan {
    std::vector<Team> teams;
    std::vector<WarpItem> witems;   // scalar teams (FP64: all teams)
    std::vector<WarpItem> witems2;  // FP32 packed same-read teams
    std::vector<CtaPair> cpairs;
    std::vector<CtaItem> citems;
    uint32_t n_long = 0, n_too_long = 0;
    double cost = 0.0;  // tuner cost model (lane-cell slots + per-row overheads)
    int N = 0;        // scalar team width (FP64: the only width)
    int NP = 0;       // packed team width (0: no packed teams)
    bool packed = false;
    int scal_id = 0;  // FP32 short-pair kernel variants (launch.h)
    int pack_id = -1;
    uint64_t bnd_words = 0;   // strip boundary buffer (tagged words)
    uint32_t n_extra = 0;     // extra partial slots (strips 1.. of wide pairs)
    int long_kind = 0;        // FP32 multi-warp kernel (launch.h: kLongN / kLongCW)
    uint32_t serial_rows = 0; // long kind 3: longest read among the serial pairs
    uint64_t wave_rows = 0;   // long kind 6: boundary rows of all strips (float4 each)
    uint64_t cells_br[3] = {0, 0, 0};  // cells of the scalar, packed and multi-warp branches
    bool fp64 = false;        // an FP64 plan (scal_id = the FP64 variant)
};

// Cost model constants (issue slots): per lane and cell of a row, and per lane and row
// (scan, shuffles, record loads, checkpoint share).
constexpr double kCellCost = 8.0;
constexpr double kRowCost = 70.0;

// Bin-pack teams (G lanes each) into 32-lane warp items within runs of similar row
// count; a warp item runs the max row count of its teams.  Appends to `teams` / `items`.
static void pack_teams(std::vector<Team>& run_teams, std::vector<uint32_t>& run_l,
                       std::vector<Team>& teams, std::vector<WarpItem>& items, double cell_w,
                       double& cost) {
    // order by l descending, then G descending
    std::vector<uint32_t> ord(run_teams.size());
    for (size_t q = 0; q < ord.size(); ++q) ord[q] = (uint32_t)q;
    std::stable_sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
        if (run_l[a] != run_l[b]) return run_l[a] > run_l[b];
        return run_teams[a].size > run_teams[b].size;
    });
    struct Bin {
        uint32_t rem, lmax;
        int32_t head, tail;
    };
    std::vector<Bin> bins;
    std::vector<Team> bt;
    std::vector<int32_t> nxt;
    std::vector<std::vector<uint32_t>> open(33);
    size_t i = 0;
    while (i < ord.size()) {
        const uint32_t l0 = run_l[ord[i]];
        size_t j = i;
        while (j < ord.size() && (double)run_l[ord[j]] >= 0.94 * (double)l0) ++j;
        std::stable_sort(ord.begin() + i, ord.begin() + j,
                         [&](uint32_t a, uint32_t b) { return run_teams[a].size > run_teams[b].size; });
        bins.clear();
        bt.clear();
        nxt.clear();
        for (auto& o : open) o.clear();
        for (size_t q = i; q < j; ++q) {
            Team t = run_teams[ord[q]];
            const uint32_t G = t.size;
            int r = -1;
            for (uint32_t c = G; c <= 32; ++c)
                if (!open[c].empty()) {
                    r = (int)c;
                    break;
                }
            uint32_t b;
            if (r < 0) {
                b = (uint32_t)bins.size();
                bins.push_back({32, 0, -1, -1});
            } else {
                b = open[r].back();
                open[r].pop_back();
            }
            t.base = (uint8_t)(32 - bins[b].rem);
            bt.push_back(t);
            nxt.push_back(-1);
            const int32_t id = (int32_t)bt.size() - 1;
            if (bins[b].tail < 0) bins[b].head = id;
            else nxt[bins[b].tail] = id;
            bins[b].tail = id;
            bins[b].rem -= G;
            bins[b].lmax = std::max(bins[b].lmax, run_l[ord[q]]);
            if (bins[b].rem > 0) open[bins[b].rem].push_back(b);
        }
        for (auto& bn : bins) {
            WarpItem w;
            w.first_team = (uint32_t)teams.size();
            w.n_teams = 0;
            for (int32_t id = bn.head; id >= 0; id = nxt[id]) {
                teams.push_back(bt[id]);
                w.n_teams++;
            }
            items.push_back(w);
            cost += (double)bn.lmax * 32.0 * (cell_w * kCellCost + kRowCost);
        }
        i = j;
    }
}

// Work plan.  Short pairs: a scalar team of G = ceil(k / Ns) lanes (k <= 32 Ns); with
// NP > 0 (FP32), two pairs of the same read with k <= 32 NP share a packed team of
// ceil(max k / NP) lanes (x / y halves).  Long pairs: W = ceil(k / (32 Nl)) warps of one
// CTA, packed best-fit into CTAs of CW warps (wider pairs: strips of CW warps).  Items
// are ordered longest first.
void make_plan(const uint32_t* l, const uint32_t* k, const uint32_t* pr, uint32_t n, int Ns, int NP,
               int Nl, Plan& P, int kw = 4, int CW = kCtaWarps, bool serial = false, bool wave = false) {
    P = Plan();
    P.N = Ns;
    P.NP = NP;
    P.packed = NP > 0;
    const uint32_t short_max = 32u * (uint32_t)Ns, packed_max = 32u * (uint32_t)NP;
    const uint32_t seg = 32u * (uint32_t)Nl;
    std::vector<uint32_t> lo;
    std::vector<Team> st, pt;  // scalar / packed teams
    std::vector<uint32_t> sl, pl;
    auto mk = [](uint32_t a, uint32_t b, uint32_t G) {
        Team t;
        t.pair = a;
        t.pair2 = b;
        t.base = 0;
        t.size = (uint8_t)G;
        t.pad = 0;
        return t;
    };
    std::vector<uint32_t> pk;  // packed-eligible pairs, grouped by read below
    for (uint32_t p = 0; p < n; ++p) {
        if (NP > 0 && k[p] <= packed_max) pk.push_back(p);
        else if (k[p] <= short_max) {
            st.push_back(mk(p, kNoPair, (k[p] + Ns - 1) / Ns));
            sl.push_back(l[p]);
        } else lo.push_back(p);
    }
    if (!pk.empty()) {
        std::stable_sort(pk.begin(), pk.end(), [&](uint32_t a, uint32_t b) {
            if (pr[a] != pr[b]) return pr[a] < pr[b];
            return k[a] > k[b];
        });
        size_t q = 0;
        while (q < pk.size()) {
            size_t e = q;
            while (e < pk.size() && pr[pk[e]] == pr[pk[q]]) ++e;
            for (; q + 1 < e; q += 2) {
                const uint32_t a = pk[q], b = pk[q + 1];
                pt.push_back(mk(a, b, (std::max(k[a], k[b]) + NP - 1) / NP));
                pl.push_back(l[a]);
            }
            if (q < e) {  // odd one out: a scalar team
                const uint32_t a = pk[q];
                st.push_back(mk(a, kNoPair, (k[a] + Ns - 1) / Ns));
                sl.push_back(l[a]);
                ++q;
            }
        }
    }
    for (const Team& t : st) P.cells_br[0] += (uint64_t)l[t.pair] * k[t.pair];
    for (const Team& t : pt)
        P.cells_br[1] += (uint64_t)l[t.pair] * k[t.pair] + (uint64_t)l[t.pair2] * k[t.pair2];
    for (uint32_t p : lo) P.cells_br[2] += (uint64_t)l[p] * k[p];
    pack_teams(st, sl, P.teams, P.witems, (double)Ns, P.cost);
    pack_teams(pt, pl, P.teams, P.witems2, 2.0 * NP * 1.2, P.cost);
    // long pairs
    P.n_long = (uint32_t)lo.size();
    auto W_of = [&](uint32_t p) { return (k[p] + seg - 1) / seg; };
    std::stable_sort(lo.begin(), lo.end(), [&](uint32_t a, uint32_t b) {
        const double ca = (double)l[a] * W_of(a), cb = (double)l[b] * W_of(b);
        return ca > cb;
    });
    auto cpair = [](uint32_t p, uint32_t w0, uint32_t W) {
        CtaPair cp;
        cp.pair = p;
        cp.w0 = (uint8_t)w0;
        cp.W = (uint8_t)W;
        cp.strip = 0;
        cp.nstrip = 1;
        cp.col0 = 0;
        cp.extra_base = 0;
        cp.pad = 0;
        cp.bnd_in = kNoBnd;
        cp.bnd_out = kNoBnd;
        return cp;
    };
    if (wave) {
        // one item per strip of 32 Nl columns, the pairs largest first and each pair's
        // strips in order, so a strip is always dequeued after the strip it waits for.
        // Strip s writes its right boundary (l float4 rows) at wave row bnd_out and
        // publishes its progress in boundary word `pad`; strip s + 1 reads both.
        for (uint32_t p : lo) {
            const uint32_t Wt = W_of(p);
            const uint32_t extra = n + P.n_extra;
            const uint64_t r0 = P.wave_rows, w0 = P.bnd_words;
            for (uint32_t stp = 0; stp < Wt; ++stp) {
                CtaPair cp = cpair(p, 0, 1);
                cp.strip = (uint16_t)stp;
                cp.nstrip = Wt;
                cp.col0 = stp * seg;
                cp.extra_base = extra;
                cp.bnd_in = stp > 0 ? r0 + (uint64_t)(stp - 1) * l[p] : kNoBnd;
                cp.bnd_out = stp + 1 < Wt ? r0 + (uint64_t)stp * l[p] : kNoBnd;
                cp.pad = (uint32_t)(w0 + stp);
                CtaItem it;
                it.first = (uint32_t)P.cpairs.size();
                it.n = 1;
                P.cpairs.push_back(cp);
                P.citems.push_back(it);
            }
            P.wave_rows += (uint64_t)(Wt - 1) * l[p];
            P.bnd_words += Wt;
            P.n_extra += Wt - 1;
            P.cost += (double)l[p] * Wt * 32.0 * (Nl * kCellCost + kRowCost);
        }
        return;
    }
    if (serial) {
        // one item per pair, largest first: a warp runs its W strips of 32 Nl columns in
        // order (strip s >= 1 leaves its partial at extra_base + s - 1)
        for (uint32_t p : lo) {
            const uint32_t Wt = W_of(p);
            CtaPair cp = cpair(p, 0, 1);
            cp.nstrip = Wt;
            if (Wt > 1) {
                cp.extra_base = n + P.n_extra;
                P.n_extra += Wt - 1;
            }
            CtaItem it;
            it.first = (uint32_t)P.cpairs.size();
            it.n = 1;
            P.cpairs.push_back(cp);
            P.citems.push_back(it);
            P.serial_rows = std::max(P.serial_rows, l[p]);
            P.cost += (double)l[p] * Wt * 32.0 * (Nl * kCellCost + kRowCost);
        }
        return;
    }
    // Units: a pair that fits one CTA, or one strip of a wider pair (S = ceil(W / CW)
    // strips of near-equal width, the wider ones first).  Units are best-fit packed into
    // CTAs of CW warps, in runs of similar read length (the CTA waits for its longest
    // unit).  A pair's strips go into bins in order, never into an earlier bin than the
    // strip before, so a strip is always dequeued no earlier than the strip it waits for
    // (the persistent kernel takes items in order: no strip waits on a strip that has not
    // been started).
    struct Unit {
        CtaPair cp;
        uint32_t l;
    };
    std::vector<Unit> units;
    for (uint32_t p : lo) {
        const uint32_t Wt = W_of(p);
        if (Wt <= (uint32_t)CW) {
            units.push_back({cpair(p, 0, Wt), l[p]});
            continue;
        }
        const uint32_t S = (Wt + CW - 1) / CW;
        const uint32_t extra = n + P.n_extra;
        const uint64_t b0 = P.bnd_words;
        uint32_t wcol = 0;
        for (uint32_t stp = 0; stp < S; ++stp) {
            const uint32_t W = Wt / S + (stp < Wt % S ? 1u : 0u);
            CtaPair cp = cpair(p, 0, W);
            cp.strip = (uint16_t)stp;
            cp.nstrip = S;
            cp.col0 = wcol * seg;
            cp.extra_base = extra;
            cp.bnd_in = stp > 0 ? b0 + (uint64_t)(stp - 1) * l[p] * kw : kNoBnd;
            cp.bnd_out = stp + 1 < S ? b0 + (uint64_t)stp * l[p] * kw : kNoBnd;
            units.push_back({cp, l[p]});
            wcol += W;
        }
        P.bnd_words += (uint64_t)(S - 1) * l[p] * kw;
        P.n_extra += S - 1;
    }
    // runs of similar length, longest first; inside a run widest first (a pair's strips
    // keep their order: their widths do not increase)
    std::stable_sort(units.begin(), units.end(), [](const Unit& x, const Unit& y) { return x.l > y.l; });
    struct CBin {
        std::vector<CtaPair> pairs;
        uint32_t rem, lmax;
    };
    std::vector<CBin> cb;
    std::vector<std::vector<uint32_t>> copen(CW + 1);
    std::vector<uint32_t> last_bin;  // per unit index of a wide pair: bin of its previous strip
    size_t a = 0;
    while (a < units.size()) {
        const uint32_t l0 = units[a].l;
        size_t b2 = a;
        while (b2 < units.size() && (double)units[b2].l >= 0.9 * (double)l0) ++b2;
        std::stable_sort(units.begin() + a, units.begin() + b2,
                         [](const Unit& x, const Unit& y) { return x.cp.W > y.cp.W; });
        cb.clear();
        for (auto& o : copen) o.clear();
        std::map<uint32_t, uint32_t> prev_bin;  // pair -> bin of its latest strip in this run
        for (size_t q = a; q < b2; ++q) {
            const Unit& u = units[q];
            const uint32_t W = u.cp.W;
            uint32_t minb = 0;
            if (u.cp.nstrip > 1) {
                auto it = prev_bin.find(u.cp.pair);
                if (it != prev_bin.end()) minb = it->second;
            }
            int r = -1;
            size_t pos = 0;
            for (uint32_t c = W; c <= (uint32_t)CW && r < 0; ++c) {
                auto& lst = copen[c];
                for (size_t z = lst.size(); z-- > 0;)
                    if (lst[z] >= minb) {
                        r = (int)c;
                        pos = z;
                        break;
                    }
            }
            uint32_t bi;
            if (r < 0) {
                bi = (uint32_t)cb.size();
                cb.push_back({{}, (uint32_t)CW, 0});
            } else {
                bi = copen[r][pos];
                copen[r].erase(copen[r].begin() + pos);
            }
            CtaPair cp = u.cp;
            cp.w0 = (uint8_t)(CW - cb[bi].rem);
            cb[bi].pairs.push_back(cp);
            cb[bi].rem -= W;
            cb[bi].lmax = std::max(cb[bi].lmax, u.l);
            if (cb[bi].rem > 0) copen[cb[bi].rem].push_back(bi);
            if (u.cp.nstrip > 1) prev_bin[u.cp.pair] = bi;
        }
        for (auto& c : cb) {
            CtaItem it;
            it.first = (uint32_t)P.cpairs.size();
            it.n = (uint32_t)c.pairs.size();
            for (auto& cp : c.pairs) P.cpairs.push_back(cp);
            P.citems.push_back(it);
            P.cost += (double)c.lmax * CW * 32.0 * (Nl * kCellCost * 1.6 + kRowCost);
        }
        a = b2;
    }
}

// ------------------------------------------------------------------------------------
// Host-side tables
// ------------------------------------------------------------------------------------
void build_phred_tables(PhredTables& T) {
    for (int x = 0; x < kPhredTab; ++x) {
        const int q = std::min(x, kMaxPhred);
        const double v = std::pow(10.0, -(double)q / 10.0);
        T.q[x] = v;
        T.om[x] = 1.0 - v;
        T.q3[x] = v / 3.0;
        T.inv[x] = 1.0 / (1.0 - v);  // inf for x = 0 (g = 1): flagged as degenerate
        T.iq[x] = std::pow(10.0, (double)q / 10.0);
    }
}

// Split power g^m (g = q(gcp)) into two factors whose product is g^m, each normal when
// g^m >= min_normal^2 (see PowRow).
template <typename T>
void split_pow(int gcp, double m, T& p1, T& p2) {
    const double lg = -(double)gcp / 10.0 * m;  // log10 of g^m
    const double min_lg = std::log10((double)std::numeric_limits<T>::min());
    if (lg >= min_lg) {
        p1 = (T)std::pow(10.0, lg);
        p2 = (T)1;
    } else {
        const double h = std::pow(10.0, lg / 2.0);
        p1 = (T)h;
        p2 = (T)h;
    }
}

template <typename T>
void build_pow_table(int N, std::vector<PowRow<T>>& out) {
    out.assign(kPhredTab, PowRow<T>());
    for (int x = 0; x < kPhredTab; ++x) {
        const int gq = std::min(x, kMaxPhred);
        PowRow<T>& r = out[x];
        for (int s = 0; s < 5; ++s) split_pow<T>(gq, (double)N * (double)(1 << s), r.sp1[s], r.sp2[s]);
        for (int t = 0; t < 32; ++t) split_pow<T>(gq, (double)N * t, r.lp1[t], r.lp2[t]);
        r.lq1[0] = r.lq2[0] = (T)0;
        for (int t = 1; t <= 32; ++t) split_pow<T>(gq, (double)N * t - 1.0, r.lq1[t], r.lq2[t]);
        split_pow<T>(gq, (double)(N / 2), r.hh1, r.hh2);
        split_pow<T>(gq, (double)(N / 2 - 1), r.hm1, r.hm2);
        split_pow<T>(gq, (double)(N - 1), r.last1, r.last2);
        r.pad1 = (T)std::pow(10.0, -(double)gq / 10.0);
        r.pad2 = (T)0;
    }
}

}  // namespace

// ------------------------------------------------------------------------------------
// Context
// ------------------------------------------------------------------------------------
struct Slot {
    DevBuf in_bases, in_bq, in_iq, in_dq, in_gq, in_hap, in_roff, in_hoff, in_pr, in_ph;
    DevBuf desc, rec32, rec32j, rec64, rec64j, teams, witems, witems2, cpairs, citems, parts, out, oflags, rescue;
    DevBuf small;  // counters[8], status[1], dropgrow[4]
    DevBuf bnd;    // strip boundaries of the batch
    DevBuf rbnd;   // rescue / launch-per-pair boundary scratch
    DevBuf sbnd;   // serial multi-warp pairs: two boundaries per resident warp
    DevBuf wbnd;   // wave multi-warp pairs: each strip's right boundary
    uint32_t sbnd_warps = 0, sbnd_rows = 0;  // what sbnd holds for the current plan
    DevBuf hdr;
    HostBuf h_out, h_oflags, h_small, h_roff, h_hoff, h_pr, h_ph;
    BatchHeader hh;
    cudaEvent_t ev_copy = nullptr, ev_start = nullptr, ev_fwd0 = nullptr, ev_fwd1 = nullptr,
                ev_res0 = nullptr, ev_res1 = nullptr, ev_end = nullptr;
    // Per-slot streams: batches in different slots run concurrently on the device.
    // sm carries the pipeline, sb2/sb3 the multi-warp and packed branches of the forward pass.
    cudaStream_t sm = nullptr, sb2 = nullptr, sb3 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join3 = nullptr, ev_user = nullptr;
    // FP32 forward branches, each timed on its own stream: [0, 1] scalar short teams (sm),
    // [2, 3] packed teams (sb3), [4, 5] multi-warp pairs (sb2)
    cudaEvent_t ev_br[6] = {};
    bool br_timed = false;
    unsigned br_mask = 0;  // branches whose events the last launch sequence recorded
    uint64_t foot = 0;  // admitted device footprint while pending
    cudaGraphExec_t gexec = nullptr;
    int g_key = -1;
    uint64_t ticket = 0;
    int state = 0;  // 0 free, 1 pending
    double* user_out = nullptr;
    uint8_t* user_flags = nullptr;
    bool out_on_dev = false;
    uint32_t n_pairs = 0;
    phmm_stats st{};
    bool has_stats = false;
    Plan plan;
    bool plan_valid = false;
    uint64_t plan_hash = 0;
    uint32_t plan_np = 0;
    int host_status = PHMM_OK;
};

struct phmm_ctx {
    int dev = 0;
    phmm_config cfg{};
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    bool own_stream = false;
    std::mutex mu;
    std::vector<Slot> slots;
    uint64_t next_ticket = 0;
    int sms = 0;
    double max_mhz = 0.0;
    size_t budget = 0;
    DevBuf tables;                          // PhredTables
    DevBuf scan_row;                        // scan test: one PowRow<float> (global memory)
    DevBuf pow32[5];                        // N = 12, 16, 20, 24 (packed short), 32 (long)
    DevBuf pow64;                           // FP64 powers, N = 8 (variant 0, rescue, comparator)
    DevBuf pow64w;                          // FP64 powers, N = 16 (variants 1-3)
    DevBuf pow64x;                          // FP64 powers, N = 32 (variant 3's short teams)
    int occ64v[kNumF64] = {1, 1, 1, 1};     // resident CTAs per SM of the FP64 forward variants
    int occ64s[kNumF64] = {1, 1, 1, 1};     // ... and of the pipelined FP64 short-team kernels
    // resident CTAs per SM of each kernel (long kind 5: resident clusters of the GPU)
    int occ_packed[kNumPacked] = {}, occ_scalar[kNumScalar] = {}, occ_longk[kNumLong] = {1, 1, 1, 1, 1, 1, 1, 1, 1}, occ64 = 1;
    std::map<uint64_t, std::array<int, 3>> tuned;  // batch signature -> (scalar id, packed id, long kind)
    uint64_t inflight_foot = 0;             // sum of pending slots' footprints
    bool dead = false;
    uint32_t seed = 0x5eed1234u;
    uint64_t last_retired = 0;
    phmm_stats last_stats{};
};

namespace {

const int kPowN[5] = {12, 16, 20, 24, 32};
int pow_index(int N) { return N == 12 ? 0 : N == 16 ? 1 : N == 20 ? 2 : N == 24 ? 3 : 4; }



#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            ctx->dead = true;                   \
            return PHMM_ECUDA;                  \
        }                                       \
    } while (0)

DevBuf* arena_bufs(Slot& S, int i) {
    DevBuf* d[] = {&S.in_bases, &S.in_bq, &S.in_iq, &S.in_dq, &S.in_gq, &S.in_hap, &S.in_roff, &S.in_hoff,
                   &S.in_pr, &S.in_ph, &S.desc, &S.rec32, &S.rec32j, &S.rec64, &S.rec64j, &S.teams, &S.witems, &S.witems2,
                   &S.cpairs, &S.citems, &S.parts, &S.out, &S.oflags, &S.rescue, &S.bnd, &S.rbnd, &S.sbnd,
                   &S.wbnd};
    return i < (int)(sizeof(d) / sizeof(d[0])) ? d[i] : nullptr;
}

uint64_t slot_capacity(Slot& S) {
    uint64_t c = 0;
    for (int i = 0; DevBuf* b = arena_bufs(S, i); ++i) c += b->cap;
    return c;
}

// Frees an idle slot's batch arenas (its header, counters and events stay).
void release_arenas(Slot& S) {
    for (int i = 0; DevBuf* b = arena_bufs(S, i); ++i) release(*b);
    S.plan_valid = false;
}

// Serial multi-warp pairs (long kind 3): two strip boundaries of serial_rows float4 rows
// for every warp of k_forward_serial's grid.
uint64_t serial_bytes(const phmm_ctx* ctx, const Plan& P) {
    if (kLongWave[P.long_kind]) return P.wave_rows * sizeof(float4);
    if (!kLongSerial[P.long_kind] || P.citems.empty()) return 0;
    const uint64_t warps = (uint64_t)ctx->sms * ctx->occ_longk[P.long_kind] * (kSerialThreads / 32);
    return warps * 2 * P.serial_rows * sizeof(float4);
}
cudaError_t ensure_serial(const phmm_ctx* ctx, Slot& S, const Plan& P) {
    if (kLongWave[P.long_kind]) {  // the wave kind's strip boundaries
        S.sbnd_warps = S.sbnd_rows = 0;
        return ensure(S.wbnd, std::max<uint64_t>(P.wave_rows, 1) * sizeof(float4));
    }
    const uint64_t b = serial_bytes(ctx, P);
    if (b == 0) {
        S.sbnd_warps = S.sbnd_rows = 0;
        return cudaSuccess;
    }
    const cudaError_t e = ensure(S.sbnd, b);
    if (e != cudaSuccess) return e;
    S.sbnd_warps = (uint32_t)ctx->sms * ctx->occ_longk[P.long_kind] * (kSerialThreads / 32);
    S.sbnd_rows = P.serial_rows;
    return cudaSuccess;
}

int launch_sequence(phmm_ctx* ctx, Slot& S, int scal_id, int pack_id, int long_kind, bool record_events) {
    cudaStream_t s = S.sm;
    const BatchHeader* H = static_cast<const BatchHeader*>(S.hdr.p);
    const PhredTables* T = static_cast<const PhredTables*>(ctx->tables.p);
    const int prec = ctx->cfg.precision;
    const int grid_pre = ctx->sms * 4;
    auto rec_on = [&](cudaEvent_t ev, cudaStream_t st) {
        if (record_events) return cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
        return cudaEventRecord(ev, st);
    };
    auto rec = [&](cudaEvent_t ev) { return rec_on(ev, s); };
    launch_reset(H, ctx->sms * 4, s);
    if (prec == PHMM_PREC_FP64) {
        // scal_id carries the FP64 variant (see make_plan64)
        launch_prep64_all(H, T, grid_pre, s);
        if (f64_pipelined(scal_id)) launch_prep64_first(H, T, grid_pre, s);
        CK(rec(S.ev_fwd0));
        const void* pw = scal_id == 0 ? ctx->pow64.p : ctx->pow64w.p;
        if (f64_pipelined(scal_id)) {
            // two branches: short teams on the pipelined engine here, multi-warp CTA items
            // on the unfactored engine on sb2
            CK(cudaEventRecord(S.ev_fork, s));
            CK(cudaStreamWaitEvent(S.sb2, S.ev_fork, 0));
            CK(rec_on(S.ev_br[4], S.sb2));
            launch_forward64(2, H, pw, ctx->sms * ctx->occ64v[2], S.sb2);
            CK(rec_on(S.ev_br[5], S.sb2));
            CK(cudaEventRecord(S.ev_join, S.sb2));
            CK(rec(S.ev_br[0]));
            launch_short_pipe64(scal_id, H, scal_id == 3 ? ctx->pow64x.p : pw, ctx->sms * ctx->occ64s[scal_id], s);
            CK(rec(S.ev_br[1]));
            CK(cudaStreamWaitEvent(s, S.ev_join, 0));
            S.br_timed = true;
            S.br_mask = 0x5u;  // no packed branch in FP64
        } else {
            launch_forward64(scal_id, H, pw, ctx->sms * ctx->occ64v[scal_id], s);
            S.br_timed = false;
        }
        CK(rec(S.ev_fwd1));
        launch_finalize64(H, grid_pre, s);
        CK(rec(S.ev_res0));
        // pairs the FP64 engine flagged (a degenerate row, range) on the unfactored engine
        launch_rescue64(H, ctx->pow64.p, ctx->sms * ctx->occ64, s);
        CK(rec(S.ev_res1));
    } else {
        launch_prep32(H, T, grid_pre, s);
        launch_prep32_first(H, T, grid_pre, s);
        CK(rec(S.ev_fwd0));
        // fork: multi-warp pairs and packed teams on two more branches, scalar teams here
        CK(cudaEventRecord(S.ev_fork, s));
        CK(cudaStreamWaitEvent(S.sb2, S.ev_fork, 0));
        CK(cudaStreamWaitEvent(S.sb3, S.ev_fork, 0));
        const void* lpow = ctx->pow32[pow_index(kLongN[long_kind])].p;
        CK(rec_on(S.ev_br[4], S.sb2));
        if (long_kind > 0)
            launch_forward32_long_pipe(long_kind, H, lpow,
                                       long_kind == 5 ? ctx->occ_longk[5] * kClusterCtas
                                                      : ctx->sms * ctx->occ_longk[long_kind],
                                       S.sb2);
        else
            launch_forward32_long(H, lpow, ctx->sms * ctx->occ_longk[0], S.sb2);
        CK(rec_on(S.ev_br[5], S.sb2));
        CK(cudaEventRecord(S.ev_join, S.sb2));
        CK(rec_on(S.ev_br[2], S.sb3));
        if (pack_id >= 0)
            launch_short_packed(pack_id, H, ctx->pow32[pow_index(kShortPackedN[pack_id])].p,
                                ctx->sms * ctx->occ_packed[pack_id], S.sb3);
        CK(rec_on(S.ev_br[3], S.sb3));
        CK(cudaEventRecord(S.ev_join3, S.sb3));
        CK(rec(S.ev_br[0]));
        launch_short_scalar(scal_id, H, ctx->pow32[pow_index(kShortScalarN[scal_id])].p,
                            ctx->sms * ctx->occ_scalar[scal_id], s);
        CK(rec(S.ev_br[1]));
        S.br_timed = true;
        S.br_mask = 0x7u;
        CK(cudaStreamWaitEvent(s, S.ev_join, 0));
        CK(cudaStreamWaitEvent(s, S.ev_join3, 0));
        CK(rec(S.ev_fwd1));
        launch_finalize32(H, grid_pre, s);
        CK(rec(S.ev_res0));
        if (prec == PHMM_PREC_FP32_RESCUE) {
            launch_prep64_list(H, T, ctx->sms * 2, s);
            launch_rescue64(H, ctx->pow64.p, ctx->sms * ctx->occ64, s);
        }
        CK(rec(S.ev_res1));
    }
    CK(cudaGetLastError());
    return PHMM_OK;
}

int kernels_per_launch(int prec, int NP, int fp64_id = 0) {
    const int packed = NP > 0 ? 1 : 0;
    // FP64: reset, prep, [first-row prep, short teams], forward, finalize, rescue
    return prec == PHMM_PREC_FP64 ? (f64_pipelined(fp64_id) ? 7 : 5) : prec == PHMM_PREC_FP32_RESCUE ? 8 + packed : 6 + packed;
}

uint64_t u64(const void* p) { return (uint64_t)(uintptr_t)p; }

// Copies a plan's arrays into the slot's device arenas (growing them as needed).
cudaError_t upload_plan(Slot& S, const Plan& P, cudaStream_t cs) {
    cudaError_t e;
    if ((e = ensure(S.teams, P.teams.size() * sizeof(Team))) != cudaSuccess) return e;
    if ((e = ensure(S.witems, P.witems.size() * sizeof(WarpItem))) != cudaSuccess) return e;
    if ((e = ensure(S.witems2, P.witems2.size() * sizeof(WarpItem))) != cudaSuccess) return e;
    if ((e = ensure(S.cpairs, P.cpairs.size() * sizeof(CtaPair))) != cudaSuccess) return e;
    if ((e = ensure(S.citems, P.citems.size() * sizeof(CtaItem))) != cudaSuccess) return e;
    auto cp = [&](DevBuf& d, const void* src, size_t n) {
        return n ? cudaMemcpyAsync(d.p, src, n, cudaMemcpyHostToDevice, cs) : cudaSuccess;
    };
    if ((e = cp(S.teams, P.teams.data(), P.teams.size() * sizeof(Team))) != cudaSuccess) return e;
    if ((e = cp(S.witems, P.witems.data(), P.witems.size() * sizeof(WarpItem))) != cudaSuccess) return e;
    if ((e = cp(S.witems2, P.witems2.data(), P.witems2.size() * sizeof(WarpItem))) != cudaSuccess) return e;
    if ((e = cp(S.cpairs, P.cpairs.data(), P.cpairs.size() * sizeof(CtaPair))) != cudaSuccess) return e;
    return cp(S.citems, P.citems.data(), P.citems.size() * sizeof(CtaItem));
}

// Plan fields of the batch header.
// The Rec32 layout is read by the lean and packed short kernels and the lean multi-warp
// kernel only; without them prep skips it and the batch needs no arena for it (an idle
// arena up to kKeepRec32Bytes is kept).
constexpr uint64_t kKeepRec32Bytes = 1ull << 30;
bool plan_needs_rec32(const Plan& P) {
    return P.pack_id >= 0 || !kShortScalarPipe[P.scal_id] || (P.long_kind == 0 && !P.citems.empty());
}

void plan_header(const Slot& S, const Plan& P, BatchHeader& hh) {
    hh.witems = (const WarpItem*)S.witems.p;
    hh.witems2 = (const WarpItem*)S.witems2.p;
    hh.n_witems2 = (uint32_t)P.witems2.size();
    hh.teams = (const Team*)S.teams.p;
    hh.citems = (const CtaItem*)S.citems.p;
    hh.cpairs = (const CtaPair*)S.cpairs.p;
    hh.n_witems = (uint32_t)P.witems.size();
    hh.n_citems = (uint32_t)P.citems.size();
    hh.n_partials = hh.n_pairs + P.n_extra;
    hh.bnd = (unsigned long long*)S.bnd.p;
    hh.n_bnd_words = P.bnd_words;
    hh.sbnd = (float4*)S.sbnd.p;
    hh.sbnd_rows = S.sbnd_rows;
    hh.sbnd_warps = S.sbnd_warps;
    hh.wbnd = (float4*)S.wbnd.p;
    if (hh.rec32 || hh.rec32j) hh.rec32 = plan_needs_rec32(P) ? (Rec32*)S.rec32.p : nullptr;
    // FP64 J-form records: only the pipelined FP64 variant reads them
    hh.rec64j = P.fp64 && f64_pipelined(P.scal_id) ? (Rec64J*)S.rec64j.p : nullptr;
}

// FP32 short-pair kernel candidates (scalar id, packed id or -1) allowed by the config.
std::vector<std::pair<int, int>> fp32_candidates(const phmm_config& cfg) {
    std::vector<std::pair<int, int>> c;
    const int v = cfg.kernel_variant, n = cfg.cols_per_lane;
    for (int si = 0; si < kNumScalar; ++si)
        for (int pi = -1; pi < kNumPacked; ++pi) {
            const bool scal_only = v >= 2;
            if (scal_only && pi >= 0) continue;
            if (v == 1 && pi < 0) continue;
            if (v == 3 && kShortScalarPipe[si]) continue;
            if (v == 4 && !kShortScalarPipe[si]) continue;
            if (v == 5 && !kShortScalarHalves[si]) continue;
            if (v == 6 && !kShortScalarLean[si]) continue;
            // the lean engine only when asked for: it measured 15% slower than the
            // three-CTA halves engine on the short-read batch (L1 reads on every row)
            if (v != 6 && kShortScalarLean[si]) continue;
            if ((n == 24 || n == 32 || n == 16) && scal_only && kShortScalarN[si] != n) continue;
            if ((n == 24 || n == 32) && !scal_only && kShortScalarN[si] != n) continue;
            if ((n == 12 || n == 16) && !scal_only && (pi < 0 || kShortPackedN[pi] != n)) continue;
            c.push_back({si, pi});
        }
    return c;
}

// FP64 plan of variant id (launch.h: kF64N columns per lane, kF64CW-warp CTAs); the
// variant travels in scal_id.
void make_plan64(const uint32_t* l, const uint32_t* k, const uint32_t* pr, uint32_t n, int id, Plan& P) {
    make_plan(l, k, pr, n, kF64NS[id], 0, kF64N[id], P, 8, kF64CW[id]);
    P.scal_id = id;
    P.pack_id = -1;
    P.long_kind = 0;
    P.fp64 = true;
    // the pipelined engine does about 6 FP64 operations per cell of a short team against
    // 8 for the unfactored one
    if (f64_pipelined(id)) P.cost -= 0.25 * (double)P.cells_br[0] * 8.0;
}

// Cluster kind: CTA items are taken kClusterCtas at a time, item g kClusterCtas + r by CTA
// rank r of a cluster.  A strip boundary whose two strips sit in neighbouring items of one
// group goes through distributed shared memory (the receiving strip's first warp in the
// marker); the others stay in global memory.
void cluster_links(Plan& P) {
    const size_t n = P.citems.size();
    for (size_t a = 0; a + 1 < n; ++a) {
        if ((a + 1) % kClusterCtas == 0) continue;  // item a + 1 starts the next group
        const CtaItem A = P.citems[a], B = P.citems[a + 1];
        for (uint32_t x = 0; x < A.n; ++x) {
            CtaPair& Lp = P.cpairs[A.first + x];
            if (Lp.bnd_out == kNoBnd) continue;
            for (uint32_t y = 0; y < B.n; ++y) {
                CtaPair& Rp = P.cpairs[B.first + y];
                if (Rp.pair == Lp.pair && Rp.strip == Lp.strip + 1) {
                    Lp.bnd_out = kDsmemBnd | Rp.w0;
                    Rp.bnd_in = kDsmemBnd;
                }
            }
        }
    }
}

void make_plan_id(const uint32_t* l, const uint32_t* k, const uint32_t* pr, uint32_t n, int scal_id,
                  int pack_id, int long_kind, Plan& P) {
    make_plan(l, k, pr, n, kShortScalarN[scal_id], pack_id >= 0 ? kShortPackedN[pack_id] : 0,
              kLongN[long_kind], P, 4, kLongCW[long_kind], kLongSerial[long_kind], kLongWave[long_kind]);
    if (long_kind == 5) cluster_links(P);
    P.scal_id = scal_id;
    P.pack_id = pack_id;
    P.long_kind = long_kind;
    // the cost model counts slots of the lean engine; the pipelined engines measured ~1.3x
    // faster per cell on every short shape
    if (!kShortScalarPipe[scal_id]) P.cost *= 1.3;
}

// FP32 multi-warp kernels the configuration allows (the lean variant keeps the lean
// engine), and the one used without measurement.
std::vector<int> long_kinds_of(const phmm_config& cfg) {
    if (cfg.flags & PHMM_F_LONG_LEAN) return {0};
    if (cfg.flags & PHMM_F_LONG_PIPE32) return {1};
    if (cfg.flags & PHMM_F_LONG_PIPE24) return {2};
    if (cfg.flags & PHMM_F_LONG_SERIAL) return {3};
    if (cfg.flags & PHMM_F_LONG_PIPE4) return {4};
    if (cfg.flags & PHMM_F_LONG_CLUSTER) return {5};
    if (cfg.flags & PHMM_F_LONG_WAVE) return {6, 7, 8};  // the wave kernels
    if (cfg.flags & PHMM_F_LONG_WAVE16) return {8};
    if (cfg.kernel_variant == 3) return {0};
    return {0, 1, 3, 4, 5, 6, 7, 8};  // kind 2 only when forced: measured slower than kind 1 everywhere
}
// Without measurement: the serial kind when multi-warp pairs outnumber the resident
// warps of k_forward_serial four times over (each warp then has several pairs to run),
// else the pipelined 12-warp kernel.
int default_long_kind(const phmm_config& cfg, uint64_t n_long = 0, uint64_t serial_warps = 0) {
    const std::vector<int> k = long_kinds_of(cfg);
    if (k.size() == 1) return k[0];
    const bool serial_ok = std::find(k.begin(), k.end(), 3) != k.end();
    if (serial_ok && serial_warps > 0 && n_long >= 4 * serial_warps) return 3;
    return std::find(k.begin(), k.end(), 1) != k.end() ? 1 : k[0];
}

// Coarse shape of a batch for the tuner cache: pair count, mean read and haplotype
// lengths (quarter-octave buckets), share of pairs whose read has other pairs.
uint64_t batch_signature(const uint32_t* l, const uint32_t* k, const uint32_t* pr, uint32_t n,
                         const phmm_config& cfg) {
    double sl = 0, sk = 0;
    uint32_t shared = 0;
    for (uint32_t p = 0; p < n; ++p) {
        sl += l[p];
        sk += k[p];
        if ((p > 0 && pr[p - 1] == pr[p]) || (p + 1 < n && pr[p + 1] == pr[p])) shared++;
    }
    auto q = [](double x) { return (uint64_t)std::max(0.0, std::floor(4.0 * std::log2(std::max(x, 1.0)))); };
    const uint64_t fs = n ? (uint64_t)(8.0 * shared / n) : 0;
    return q(n) | (q(sl / std::max(n, 1u)) << 8) | (q(sk / std::max(n, 1u)) << 16) | (fs << 24) |
           ((uint64_t)cfg.precision << 32) | ((uint64_t)cfg.kernel_variant << 36) |
           ((uint64_t)cfg.cols_per_lane << 40);
}

constexpr uint64_t kTuneMinCells = 200000000ull;  // smaller batches keep the cost model's pick

}  // namespace

extern "C" {

int phmm_abi_version(void) { return PHMM_ABI_VERSION; }

const char* phmm_strerror(int s) {
    switch (s) {
    case PHMM_OK: return "ok";
    case PHMM_PENDING: return "pending";
    case PHMM_EINVAL: return "invalid argument or input";
    case PHMM_ENOMEM: return "batch exceeds the device memory budget";
    case PHMM_EBUSY: return "too many batches in flight";
    case PHMM_ECUDA: return "CUDA error";
    case PHMM_ETIMEOUT: return "timed out";
    case PHMM_ECANCELED: return "cancelled";
    case PHMM_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
    }
}

int phmm_create(const phmm_config* cfg, phmm_ctx** out) {
    if (!cfg || !out) return PHMM_EINVAL;
    *out = nullptr;
    if (cfg->precision < 0 || cfg->precision > 2) return PHMM_EINVAL;
    if (cfg->kernel_variant < 0 || cfg->kernel_variant > 6) return PHMM_EINVAL;
    if (!(cfg->fp32_tolerance >= 0.0)) return PHMM_EINVAL;
    {
        const unsigned lk =
            cfg->flags & (PHMM_F_LONG_LEAN | PHMM_F_LONG_PIPE32 | PHMM_F_LONG_PIPE24 | PHMM_F_LONG_SERIAL |
                          PHMM_F_LONG_PIPE4 | PHMM_F_LONG_CLUSTER | PHMM_F_LONG_WAVE | PHMM_F_LONG_WAVE16);
        if (lk & (lk - 1)) return PHMM_EINVAL;  // more than one forced multi-warp kernel
    }
    {
        const int n = cfg->cols_per_lane;
        const bool okp = n == 12 || n == 16;  // packed widths
        const bool oks = n == 16 || n == 24 || n == 32;  // scalar widths
        if (cfg->precision == PHMM_PREC_FP64) {
            if (n != 0 && n != kF64N[0] && n != kF64N[1]) return PHMM_EINVAL;  // the FP64 variants
        } else if (n != 0 && !(cfg->kernel_variant >= 2 ? oks : (okp || oks))) {
            return PHMM_EINVAL;
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
        return PHMM_ECUDA;
    phmm_ctx* ctx = new phmm_ctx();
    ctx->dev = cfg->device;
    ctx->cfg = *cfg;
    if (ctx->cfg.max_inflight == 0) ctx->cfg.max_inflight = 4;
    if (ctx->cfg.max_inflight > 64) ctx->cfg.max_inflight = 64;
    auto fail = [&](int code) {
        phmm_destroy(ctx);
        return code;
    };
    if (cudaSetDevice(ctx->dev) != cudaSuccess) return fail(PHMM_ECUDA);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->dev);
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->dev);
    ctx->max_mhz = khz / 1000.0;
    if (cfg->stream) {
        ctx->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(PHMM_ECUDA);
        ctx->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(PHMM_ECUDA);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    ctx->budget = cfg->mem_budget_bytes ? cfg->mem_budget_bytes : (size_t)(0.9 * (double)fr);
    // tables
    PhredTables T;
    build_phred_tables(T);
    if (ensure(ctx->tables, sizeof(T)) != cudaSuccess) return fail(PHMM_ECUDA);
    cudaMemcpy(ctx->tables.p, &T, sizeof(T), cudaMemcpyHostToDevice);
    for (int q = 0; q < 5; ++q) {
        std::vector<PowRow<float>> v;
        build_pow_table<float>(kPowN[q], v);
        if (ensure(ctx->pow32[q], v.size() * sizeof(v[0])) != cudaSuccess) return fail(PHMM_ECUDA);
        cudaMemcpy(ctx->pow32[q].p, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
    }
    for (int q = 0; q < kNumPacked; ++q) ctx->occ_packed[q] = occupancy_short_packed(q);
    for (int q = 0; q < kNumScalar; ++q) ctx->occ_scalar[q] = occupancy_short_scalar(q);
    ctx->occ_longk[0] = occupancy_forward32_long();
    ctx->occ_longk[1] = occupancy_forward32_long_pipe(1);
    ctx->occ_longk[2] = occupancy_forward32_long_pipe(2);
    ctx->occ_longk[3] = occupancy_forward32_long_pipe(3);
    ctx->occ_longk[4] = occupancy_forward32_long_pipe(4);
    ctx->occ_longk[5] = occupancy_forward32_long_pipe(5);
    ctx->occ_longk[6] = occupancy_forward32_long_pipe(6);
    ctx->occ_longk[7] = occupancy_forward32_long_pipe(7);
    ctx->occ_longk[8] = occupancy_forward32_long_pipe(8);
    if (getenv("PHMM_DEBUG")) {
        fprintf(stderr, "phmm: sms %d occupancy packed %d %d long %d %d %d %d %d fp64 %d scalar", ctx->sms,
                ctx->occ_packed[0], ctx->occ_packed[1], ctx->occ_longk[0], ctx->occ_longk[1],
                ctx->occ_longk[2], ctx->occ_longk[3], ctx->occ_longk[4], ctx->occ64);
        for (int q = 0; q < kNumScalar; ++q) fprintf(stderr, " %d", ctx->occ_scalar[q]);
        fprintf(stderr, "\n");
    }
    {
        std::vector<PowRow<double>> v;
        build_pow_table<double>(kN64, v);
        if (ensure(ctx->pow64, v.size() * sizeof(v[0])) != cudaSuccess) return fail(PHMM_ECUDA);
        cudaMemcpy(ctx->pow64.p, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
        build_pow_table<double>(kF64N[1], v);
        if (ensure(ctx->pow64w, v.size() * sizeof(v[0])) != cudaSuccess) return fail(PHMM_ECUDA);
        cudaMemcpy(ctx->pow64w.p, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
        build_pow_table<double>(kF64NS[3], v);
        if (ensure(ctx->pow64x, v.size() * sizeof(v[0])) != cudaSuccess) return fail(PHMM_ECUDA);
        cudaMemcpy(ctx->pow64x.p, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
        for (int q = 0; q < kNumF64; ++q) ctx->occ64v[q] = occupancy_forward64(q);
        for (int q = 2; q < kNumF64; ++q) ctx->occ64s[q] = occupancy_short_pipe64(q);
        ctx->occ64 = ctx->occ64v[0];
    }
    ctx->slots.resize(ctx->cfg.max_inflight);
    for (auto& S : ctx->slots) {
        cudaEvent_t* evs[] = {&S.ev_copy, &S.ev_start, &S.ev_fwd0, &S.ev_fwd1, &S.ev_res0, &S.ev_res1, &S.ev_end,
                              &S.ev_br[0], &S.ev_br[1], &S.ev_br[2], &S.ev_br[3], &S.ev_br[4], &S.ev_br[5]};
        for (auto* e : evs)
            if (cudaEventCreate(e) != cudaSuccess) return fail(PHMM_ECUDA);
        cudaEvent_t* evn[] = {&S.ev_fork, &S.ev_join, &S.ev_join3, &S.ev_user};
        for (auto* e : evn)
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return fail(PHMM_ECUDA);
        cudaStream_t* sts[] = {&S.sm, &S.sb2, &S.sb3};
        for (auto* q : sts)
            if (cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess) return fail(PHMM_ECUDA);
        if (ensure(S.small, 64) != cudaSuccess || ensure(S.h_small, 64) != cudaSuccess ||
            ensure(S.hdr, sizeof(BatchHeader)) != cudaSuccess)
            return fail(PHMM_ECUDA);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(PHMM_ECUDA);
    *out = ctx;
    return PHMM_OK;
}

void phmm_destroy(phmm_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    for (auto& S : ctx->slots) {
        cudaStream_t sts[] = {S.sm, S.sb2, S.sb3};
        for (auto q : sts)
            if (q) cudaStreamSynchronize(q);
    }
    for (auto& S : ctx->slots) {
        DevBuf* d[] = {&S.in_bases, &S.in_bq, &S.in_iq, &S.in_dq, &S.in_gq, &S.in_hap, &S.in_roff,
                       &S.in_hoff, &S.in_pr, &S.in_ph, &S.desc, &S.rec32, &S.rec32j, &S.rec64, &S.rec64j, &S.teams,
                       &S.witems, &S.witems2, &S.cpairs, &S.citems, &S.parts, &S.out, &S.oflags, &S.rescue,
                       &S.small, &S.hdr, &S.bnd, &S.rbnd, &S.sbnd, &S.wbnd};
        for (auto* b : d) release(*b);
        HostBuf* h[] = {&S.h_out, &S.h_oflags, &S.h_small, &S.h_roff, &S.h_hoff, &S.h_pr, &S.h_ph};
        for (auto* b : h) release(*b);
        cudaEvent_t evs[] = {S.ev_copy, S.ev_start, S.ev_fwd0, S.ev_fwd1, S.ev_res0, S.ev_res1, S.ev_end,
                             S.ev_br[0], S.ev_br[1], S.ev_br[2], S.ev_br[3], S.ev_br[4], S.ev_br[5]};
        for (auto e : evs)
            if (e) cudaEventDestroy(e);
        cudaEvent_t evn[] = {S.ev_fork, S.ev_join, S.ev_join3, S.ev_user};
        for (auto e : evn)
            if (e) cudaEventDestroy(e);
        if (S.gexec) cudaGraphExecDestroy(S.gexec);
        cudaStream_t sts[] = {S.sm, S.sb2, S.sb3};
        for (auto q : sts)
            if (q) cudaStreamDestroy(q);
    }
    release(ctx->tables);
    release(ctx->scan_row);
    for (auto& b : ctx->pow32) release(b);
    release(ctx->pow64);
    release(ctx->pow64w);
    release(ctx->pow64x);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int phmm_device_info(phmm_ctx* ctx, int* sms, double* max_clock_mhz, double* cups) {
    if (!ctx) return PHMM_EINVAL;
    if (sms) *sms = ctx->sms;
    if (max_clock_mhz) *max_clock_mhz = ctx->max_mhz;
    if (cups) *cups = 2.0 * 128.0 * ctx->sms * ctx->max_mhz * 1e6 / 12.0;
    return PHMM_OK;
}

int phmm_submit_batch(phmm_ctx* ctx, const phmm_batch* b, uint64_t* ticket) {
    if (!ctx || !b || !ticket) return PHMM_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->dead) return PHMM_ECUDA;
    if (cudaSetDevice(ctx->dev) != cudaSuccess) return PHMM_ECUDA;
    if (b->n_pairs > 0 && (!b->read_bases || !b->read_off || !b->base_q || !b->ins_q || !b->del_q ||
                           !b->gcp_q || !b->hap_bases || !b->hap_off || !b->pair_read ||
                           !b->pair_hap || !b->out_log10))
        return PHMM_EINVAL;
    if (b->n_pairs > 0 && (b->n_reads == 0 || b->n_haps == 0)) return PHMM_EINVAL;
    // a free slot
    Slot* S = nullptr;
    for (auto& s : ctx->slots)
        if (s.state == 0) {
            S = &s;
            break;
        }
    if (!S) return PHMM_EBUSY;
    const bool dev_in = b->inputs_on_device != 0;
    const uint32_t nr = b->n_reads, nh = b->n_haps, np = b->n_pairs;
    // host views of offsets and the pair index
    const uint64_t *roff = b->read_off, *hoff = b->hap_off;
    const uint32_t *pr = b->pair_read, *ph = b->pair_hap;
    if (dev_in && np > 0) {
        // device inputs are produced on the caller's stream: read them after its pending work
        CK(cudaEventRecord(S->ev_user, ctx->stream));
        CK(cudaStreamWaitEvent(ctx->copy_stream, S->ev_user, 0));
        CK(ensure(S->h_roff, (nr + 1) * 8ull));
        CK(ensure(S->h_hoff, (nh + 1) * 8ull));
        CK(ensure(S->h_pr, np * 4ull));
        CK(ensure(S->h_ph, np * 4ull));
        CK(cudaMemcpyAsync(S->h_roff.p, b->read_off, (nr + 1) * 8ull, cudaMemcpyDeviceToHost, ctx->copy_stream));
        CK(cudaMemcpyAsync(S->h_hoff.p, b->hap_off, (nh + 1) * 8ull, cudaMemcpyDeviceToHost, ctx->copy_stream));
        CK(cudaMemcpyAsync(S->h_pr.p, b->pair_read, np * 4ull, cudaMemcpyDeviceToHost, ctx->copy_stream));
        CK(cudaMemcpyAsync(S->h_ph.p, b->pair_hap, np * 4ull, cudaMemcpyDeviceToHost, ctx->copy_stream));
        CK(cudaStreamSynchronize(ctx->copy_stream));
        roff = static_cast<const uint64_t*>(S->h_roff.p);
        hoff = static_cast<const uint64_t*>(S->h_hoff.p);
        pr = static_cast<const uint32_t*>(S->h_pr.p);
        ph = static_cast<const uint32_t*>(S->h_ph.p);
    }
    // validation: offsets non-decreasing with lengths >= 1, indices in range
    std::vector<uint32_t> L(np), K(np);
    uint64_t cells = 0;
    if (np > 0) {
        if (roff[0] != 0 || hoff[0] != 0) return PHMM_EINVAL;
        for (uint32_t r = 0; r < nr; ++r)
            if (roff[r + 1] <= roff[r] || roff[r + 1] - roff[r] > 0xffffffull) return PHMM_EINVAL;
        for (uint32_t h = 0; h < nh; ++h)
            if (hoff[h + 1] <= hoff[h] || hoff[h + 1] - hoff[h] > 0xffffffull) return PHMM_EINVAL;
        for (uint32_t p = 0; p < np; ++p) {
            if (pr[p] >= nr || ph[p] >= nh) return PHMM_EINVAL;
            L[p] = (uint32_t)(roff[pr[p] + 1] - roff[pr[p]]);
            K[p] = (uint32_t)(hoff[ph[p] + 1] - hoff[ph[p]]);
            cells += (uint64_t)L[p] * K[p];
        }
    }
    const uint64_t nbases = np > 0 ? roff[nr] : 0, nhb = np > 0 ? hoff[nh] : 0;
    // plan (FP32: packed short width from the config or the cost model; FP64: kN64).
    // A batch with the same pair lengths as this slot's previous one reuses its plan.
    const auto th0 = std::chrono::steady_clock::now();
    uint64_t hsh = 1469598103934665603ull ^ ((uint64_t)ctx->cfg.precision << 32) ^ (uint64_t)ctx->cfg.cols_per_lane ^ ((uint64_t)ctx->cfg.kernel_variant << 40);
    for (uint32_t p = 0; p < np; ++p) {
        hsh = (hsh ^ ((uint64_t)L[p] << 24 ^ K[p])) * 1099511628211ull;
    }
    hsh ^= np;
    Plan& P = S->plan;
    int N = kN64;
    bool tune_short = false, tune_long = false, tune64 = false;
    uint64_t tune_sig = 0;
    std::vector<std::pair<int, int>> tune_cand;
    const bool reuse = S->plan_valid && S->plan_hash == hsh && S->plan_np == np;
    if (!reuse) {
        if (ctx->cfg.precision == PHMM_PREC_FP64) {
            // FP64 variant: cached choice for this batch shape, else the cost model's (the
            // smaller plan cost), measured below for large batches
            const uint64_t sig = batch_signature(L.data(), K.data(), pr, np, ctx->cfg);
            auto hit = ctx->tuned.find(sig);
            // forced: cols_per_lane 8 / 16 = the unfactored variants, kernel_variant 4 (the
            // pipelined engine, 16-column teams) = variant 2, 5 or 6 (32-column fused
            // teams) = variant 3
            const int forced = ctx->cfg.kernel_variant >= 5 ? 3 : ctx->cfg.kernel_variant == 4 ? 2
                             : ctx->cfg.cols_per_lane == kF64N[0] ? 0
                             : ctx->cfg.cols_per_lane == kF64N[1] ? 1 : -1;
            if (forced >= 0) {
                make_plan64(L.data(), K.data(), pr, np, forced, P);
            } else if (hit != ctx->tuned.end()) {
                make_plan64(L.data(), K.data(), pr, np, hit->second[0], P);
            } else {
                make_plan64(L.data(), K.data(), pr, np, 0, P);
                for (int id = 1; id < kNumF64; ++id) {
                    Plan c;
                    make_plan64(L.data(), K.data(), pr, np, id, c);
                    if (c.cost < P.cost) P = std::move(c);
                }
                tune64 = !(ctx->cfg.flags & PHMM_F_NO_TUNE) && !(ctx->cfg.flags & PHMM_F_LAUNCH_PER_PAIR) &&
                         cells >= kTuneMinCells;
                tune_sig = sig;
            }
        } else {
            const std::vector<std::pair<int, int>> cand = fp32_candidates(ctx->cfg);
            const uint64_t sig = batch_signature(L.data(), K.data(), pr, np, ctx->cfg);
            auto hit = ctx->tuned.find(sig);
            if (hit != ctx->tuned.end()) {
                make_plan_id(L.data(), K.data(), pr, np, hit->second[0], hit->second[1], hit->second[2], P);
            } else {
                // cost-model choice first; measured tuning (below) may replace it
                uint64_t n_wide = 0;  // pairs wider than one warp of 32 columns per lane
                for (uint32_t p = 0; p < np; ++p) n_wide += K[p] > 1024u;
                const int dlk = default_long_kind(ctx->cfg, n_wide,
                                                  (uint64_t)ctx->sms * ctx->occ_longk[3] * (kSerialThreads / 32));
                Plan best;
                bool have = false;
                for (auto& cd : cand) {
                    Plan c;
                    make_plan_id(L.data(), K.data(), pr, np, cd.first, cd.second, dlk, c);
                    const double cost = c.cost + (double)c.n_too_long * 1e18;
                    if (!have || cost < best.cost + (double)best.n_too_long * 1e18) {
                        best = std::move(c);
                        have = true;
                    }
                }
                P = std::move(best);
                // measure the short-pair kernels when short pairs, and the multi-warp
                // kernels when multi-warp pairs, hold a real share of the batch's cells
                uint64_t short_cells = 0;
                const uint64_t wmax = 32ull * 32ull;  // widest short team: 32 lanes x 32 columns
                for (uint32_t p = 0; p < np; ++p)
                    if (K[p] <= wmax) short_cells += (uint64_t)L[p] * K[p];
                const uint64_t long_cells = cells - short_cells;
                const bool may_tune = !(ctx->cfg.flags & PHMM_F_NO_TUNE);
                tune_short = may_tune && cand.size() > 1 && short_cells >= kTuneMinCells && short_cells * 10 >= cells;
                tune_long = may_tune && long_kinds_of(ctx->cfg).size() > 1 && long_cells >= kTuneMinCells &&
                            long_cells * 10 >= cells;
                tune_sig = sig;
                tune_cand = cand;
            }
        }
    }
    N = P.N;
    const auto th_plan = std::chrono::steady_clock::now();
    // footprint and admission (lean records only for a plan that reads them, or for the
    // tuner's trials, which may)
    const bool need64 = ctx->cfg.precision != PHMM_PREC_FP32_ONLY;
    const bool need32 = ctx->cfg.precision != PHMM_PREC_FP64 &&
                        (tune_short || tune_long || plan_needs_rec32(P));
    uint32_t lmax_b = 0;
    for (uint32_t p = 0; p < np; ++p) lmax_b = std::max(lmax_b, L[p]);
    const uint64_t rb_words = (uint64_t)lmax_b * 8;  // FP64 boundary: 8 words per row
    const int rescue_ctas = ctx->sms * ctx->occ64;
    const uint64_t rb_bytes = (uint64_t)rescue_ctas * 2 * rb_words * 8ull + 16;
    const uint64_t foot = (dev_in ? 0 : nbases * 5 + nhb + (nr + 1) * 8ull + (nh + 1) * 8ull + np * 8ull) +
                          (ctx->cfg.precision != PHMM_PREC_FP32_ONLY ? rb_bytes : 0) +
                          np * (sizeof(PairDesc) + sizeof(Partial) + 8 + 1 + 4) +
                          (ctx->cfg.precision == PHMM_PREC_FP64 ? 0 : nbases * sizeof(Rec32J)) +
                          (need32 ? nbases * sizeof(Rec32) : 0) +
                          (need64 ? nbases * sizeof(Rec64) : 0) +
                          (ctx->cfg.precision == PHMM_PREC_FP64 ? nbases * sizeof(Rec64J) : 0) +
                          P.teams.size() * sizeof(Team) + (P.witems.size() + P.witems2.size()) * sizeof(WarpItem) +
                          P.cpairs.size() * sizeof(CtaPair) + P.citems.size() * sizeof(CtaItem) +
                          P.bnd_words * 8ull + P.n_extra * sizeof(Partial) + serial_bytes(ctx, P);
    if (foot > ctx->budget) return PHMM_ENOMEM;
    if (foot + ctx->inflight_foot > ctx->budget) return PHMM_EBUSY;  // admissible once others retire
    {
        // arenas persist across batches; give back idle slots' arenas when the budget needs them
        uint64_t held = 0;
        for (auto& o : ctx->slots)
            if (&o != S) held += slot_capacity(o);
        if (held + std::max<uint64_t>(foot, slot_capacity(*S)) > ctx->budget)
            for (auto& o : ctx->slots)
                if (&o != S && o.state == 0) release_arenas(o);
    }
    // device arenas
    BatchHeader& hh = S->hh;
    memset(&hh, 0, sizeof(hh));
    if (dev_in) {
        hh.read_bases = b->read_bases; hh.base_q = b->base_q; hh.ins_q = b->ins_q;
        hh.del_q = b->del_q; hh.gcp_q = b->gcp_q; hh.hap_bases = b->hap_bases;
        hh.read_off = b->read_off; hh.hap_off = b->hap_off;
        hh.pair_read = b->pair_read; hh.pair_hap = b->pair_hap;
    } else if (np > 0) {
        CK(ensure(S->in_bases, nbases)); CK(ensure(S->in_bq, nbases)); CK(ensure(S->in_iq, nbases));
        CK(ensure(S->in_dq, nbases)); CK(ensure(S->in_gq, nbases)); CK(ensure(S->in_hap, nhb));
        CK(ensure(S->in_roff, (nr + 1) * 8ull)); CK(ensure(S->in_hoff, (nh + 1) * 8ull));
        CK(ensure(S->in_pr, np * 4ull)); CK(ensure(S->in_ph, np * 4ull));
        cudaStream_t cs = ctx->copy_stream;
        CK(cudaMemcpyAsync(S->in_bases.p, b->read_bases, nbases, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_bq.p, b->base_q, nbases, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_iq.p, b->ins_q, nbases, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_dq.p, b->del_q, nbases, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_gq.p, b->gcp_q, nbases, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_hap.p, b->hap_bases, nhb, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_roff.p, b->read_off, (nr + 1) * 8ull, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_hoff.p, b->hap_off, (nh + 1) * 8ull, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_pr.p, b->pair_read, np * 4ull, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(S->in_ph.p, b->pair_hap, np * 4ull, cudaMemcpyHostToDevice, cs));
        if (getenv("PHMM_DEBUG"))
            fprintf(stderr, "phmm submit: input copies issued %.1f ms after the plan\n",
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th_plan).count());
        hh.read_bases = (const uint8_t*)S->in_bases.p; hh.base_q = (const uint8_t*)S->in_bq.p;
        hh.ins_q = (const uint8_t*)S->in_iq.p; hh.del_q = (const uint8_t*)S->in_dq.p;
        hh.gcp_q = (const uint8_t*)S->in_gq.p; hh.hap_bases = (const uint8_t*)S->in_hap.p;
        hh.read_off = (const uint64_t*)S->in_roff.p; hh.hap_off = (const uint64_t*)S->in_hoff.p;
        hh.pair_read = (const uint32_t*)S->in_pr.p; hh.pair_hap = (const uint32_t*)S->in_ph.p;
    }
    CK(ensure(S->desc, np * sizeof(PairDesc)));
    if (ctx->cfg.precision != PHMM_PREC_FP64) {
        // a large arena this plan does not read (e.g. left from the tuner's trials) goes
        // back; a small one stays, so that batches alternating between plans that read it
        // and plans that do not pay no cudaFree (a device-wide synchronisation) each time
        if (need32) CK(ensure(S->rec32, nbases * sizeof(Rec32)));
        else if (S->rec32.cap > kKeepRec32Bytes) release(S->rec32);
        CK(ensure(S->rec32j, nbases * sizeof(Rec32J)));
    }
    if (need64) CK(ensure(S->rec64, nbases * sizeof(Rec64)));
    if (ctx->cfg.precision == PHMM_PREC_FP64) CK(ensure(S->rec64j, nbases * sizeof(Rec64J)));
    CK(ensure(S->parts, (np + P.n_extra) * sizeof(Partial)));
    CK(ensure(S->bnd, P.bnd_words * 8ull));
    CK(ensure_serial(ctx, *S, P));
    if (ctx->cfg.precision != PHMM_PREC_FP32_ONLY) CK(ensure(S->rbnd, rb_bytes));
    CK(ensure(S->out, np * 8ull));
    CK(ensure(S->oflags, np * 1ull));
    CK(ensure(S->rescue, np * 4ull));
    CK(ensure(S->h_out, np * 8ull));
    CK(ensure(S->h_oflags, np * 1ull));
    cudaStream_t cs = ctx->copy_stream;
    if (!reuse) CK(upload_plan(*S, P, cs));
    CK(cudaMemsetAsync(S->parts.p, 0, (np + P.n_extra) * sizeof(Partial), cs));
    hh.n_read_bases = nbases;
    hh.n_reads = nr;
    hh.n_haps = nh;
    hh.n_pairs = np;
    hh.desc = (PairDesc*)S->desc.p;
    hh.rec32 = (Rec32*)S->rec32.p;
    hh.rec32j = ctx->cfg.precision != PHMM_PREC_FP64 ? (Rec32J*)S->rec32j.p : nullptr;
    hh.rec64 = (Rec64*)S->rec64.p;
    plan_header(*S, P, hh);
    hh.n_partials = np + P.n_extra;
    hh.bnd = (unsigned long long*)S->bnd.p;
    hh.n_bnd_words = P.bnd_words;
    hh.rbnd = (unsigned long long*)S->rbnd.p;
    hh.rbnd_words_per_cta = rb_words;
    hh.l_max = lmax_b;
    hh.force_rescue = (ctx->cfg.flags & PHMM_F_FORCE_RESCUE) ? 1u : 0u;
    hh.tol32 = ctx->cfg.fp32_tolerance > 0.0 ? ctx->cfg.fp32_tolerance : 1e-3;
    hh.parts = (Partial*)S->parts.p;
    hh.out = (double*)S->out.p;
    hh.out_flags = (uint8_t*)S->oflags.p;
    hh.rescue_list = (uint32_t*)S->rescue.p;
    hh.counters = (uint32_t*)S->small.p;          // words 0..7
    hh.status = (uint32_t*)S->small.p + 8;        // word 8
    hh.dropgrow = (uint32_t*)S->small.p + 9;      // words 9 .. 12
    hh.seed = ctx->seed;
    hh.mode = (uint32_t)ctx->cfg.precision;
    CK(cudaMemcpyAsync(S->hdr.p, &hh, sizeof(hh), cudaMemcpyHostToDevice, cs));
    CK(cudaEventRecord(S->ev_copy, cs));
    // host inputs may be released when submit returns
    CK(cudaEventSynchronize(S->ev_copy));
    // this slot's pipeline runs after the caller's pending work and the uploads
    CK(cudaEventRecord(S->ev_user, ctx->stream));
    CK(cudaStreamWaitEvent(S->sm, S->ev_user, 0));
    CK(cudaStreamWaitEvent(S->sm, S->ev_copy, 0));
    if (tune64) {
        // Measured choice of the FP64 variant: the forward pass of each, twice (the first
        // launch after a plan change runs cold), the faster kept for this batch shape.
        float best_ms = 1e30f;
        int best = P.scal_id;
        for (int id = 0; id < kNumF64; ++id) {
            Plan c;
            make_plan64(L.data(), K.data(), pr, np, id, c);
            if (c.n_too_long) continue;
            CK(upload_plan(*S, c, cs));
            CK(ensure(S->parts, (np + c.n_extra) * sizeof(Partial)));
            CK(ensure(S->bnd, c.bnd_words * 8ull));
            hh.parts = (Partial*)S->parts.p;
            plan_header(*S, c, hh);
            CK(cudaMemcpyAsync(S->hdr.p, &hh, sizeof(hh), cudaMemcpyHostToDevice, cs));
            CK(cudaStreamSynchronize(cs));
            float ms = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                const int rc = launch_sequence(ctx, *S, id, -1, 0, false);
                if (rc != PHMM_OK) return rc;
                CK(cudaStreamSynchronize(S->sm));
                float m1 = 0.f;
                CK(cudaEventElapsedTime(&m1, S->ev_fwd0, S->ev_fwd1));
                ms = std::min(ms, m1);
                if (m1 > 100.f) break;
            }
            if (getenv("PHMM_DEBUG"))
                fprintf(stderr, "phmm tuner: fp64 variant %d (N %d/%d, %d-warp CTAs): forward %.3f ms\n", id, kF64NS[id], kF64N[id],
                        kF64CW[id], ms);
            if (ms < best_ms) {
                best_ms = ms;
                best = id;
            }
        }
        ctx->tuned[tune_sig] = {best, -1, 0};
        make_plan64(L.data(), K.data(), pr, np, best, P);
        CK(upload_plan(*S, P, cs));
        CK(ensure(S->parts, (np + P.n_extra) * sizeof(Partial)));
        CK(ensure(S->bnd, P.bnd_words * 8ull));
        hh.parts = (Partial*)S->parts.p;
        plan_header(*S, P, hh);
        CK(cudaMemcpyAsync(S->hdr.p, &hh, sizeof(hh), cudaMemcpyHostToDevice, cs));
        CK(cudaMemsetAsync(S->parts.p, 0, (np + P.n_extra) * sizeof(Partial), cs));
        CK(cudaStreamSynchronize(cs));
    }
    if (tune_short || tune_long) {
        // Measured tuning: run the FP32 pipeline once per candidate on this batch (events
        // around the forward kernels), keep the fastest for this shape: first the short-
        // pair kernels, then the multi-warp kernel.
        cudaStream_t ts = S->sm;
        double best_ms = 1e30;
        int bs = P.scal_id, bp = P.pack_id, bl = P.long_kind;
        std::vector<std::array<int, 3>> runs;
        if (tune_short)
            for (auto& cd : tune_cand) runs.push_back({cd.first, cd.second, bl});
        const size_t n_short = runs.size();
        if (tune_long) {
            // the serial kind needs about one multi-warp pair per resident warp or more:
            // with far fewer it leaves most of the GPU idle, so it is not worth a (long)
            // trial run (at half as many pairs as warps it can still win: measured)
            const uint64_t swarps = (uint64_t)ctx->sms * ctx->occ_longk[3] * (kSerialThreads / 32);
            // the 4-warp-CTA kind pays off only for a few very wide pairs (it spreads them over
            // more SMs); with many wide pairs it is not worth a trial run either
            for (int lk : long_kinds_of(ctx->cfg)) {
                if (kLongSerial[lk] && 2 * (uint64_t)P.n_long < swarps) continue;
                if ((lk == 4 || lk == 5 || kLongWave[lk]) && (uint64_t)P.n_long >= swarps) continue;
                runs.push_back({-1, -1, lk});
            }
        }
        for (size_t ri = 0; ri < runs.size(); ++ri) {
            if (ri == n_short) best_ms = 1e30;  // second stage: the short choice is fixed
            std::array<int, 3> cd = runs[ri];
            if (cd[0] < 0) {
                cd[0] = bs;
                cd[1] = bp;
            }
            Plan c;
            make_plan_id(L.data(), K.data(), pr, np, cd[0], cd[1], cd[2], c);
            if (c.n_too_long) continue;
            CK(upload_plan(*S, c, cs));
            CK(ensure(S->parts, (np + c.n_extra) * sizeof(Partial)));
            CK(ensure(S->bnd, c.bnd_words * 8ull));
            CK(ensure_serial(ctx, *S, c));
            hh.parts = (Partial*)S->parts.p;
            plan_header(*S, c, hh);
            CK(cudaMemcpyAsync(S->hdr.p, &hh, sizeof(hh), cudaMemcpyHostToDevice, cs));
            CK(cudaStreamSynchronize(cs));
            // time the candidate; a short run is repeated and the faster kept (the first
            // launch of a kernel after a plan change runs cold).  The serial multi-warp kind
            // is always run twice: its first run after a plan change measured about 30%
            // slower than its steady state, which would bias the choice against it.
            float ms = 1e30f, first = 0.f;
            const bool warm_twice = !c.citems.empty() && kLongSerial[c.long_kind];
            for (int rep = 0; rep < 2; ++rep) {
                const int rc = launch_sequence(ctx, *S, c.scal_id, c.pack_id, c.long_kind, false);
                if (rc != PHMM_OK) return rc;
                CK(cudaStreamSynchronize(ts));
                float m1 = 0.f;
                CK(cudaEventElapsedTime(&m1, S->ev_fwd0, S->ev_fwd1));
                if (rep == 0) first = m1;
                ms = std::min(ms, m1);
                if (m1 > 100.f && !(warm_twice && rep == 0)) break;
            }
            if (getenv("PHMM_DEBUG"))
                fprintf(stderr, "phmm tuner: scalar %d (N %d%s) packed %d long %d: forward %.3f ms (first run %.3f)\n",
                        cd[0], kShortScalarN[cd[0]], kShortScalarPipe[cd[0]] ? " pipelined" : "", cd[1], cd[2], ms,
                        first);
            if (ms < best_ms) {
                best_ms = ms;
                bs = cd[0];
                bp = cd[1];
                bl = cd[2];
            }
        }
        ctx->tuned[tune_sig] = {bs, bp, bl};
        make_plan_id(L.data(), K.data(), pr, np, bs, bp, bl, P);
        CK(upload_plan(*S, P, cs));
        CK(ensure(S->parts, (np + P.n_extra) * sizeof(Partial)));
        CK(ensure(S->bnd, P.bnd_words * 8ull));
        CK(ensure_serial(ctx, *S, P));
        hh.parts = (Partial*)S->parts.p;
        plan_header(*S, P, hh);
        CK(cudaMemcpyAsync(S->hdr.p, &hh, sizeof(hh), cudaMemcpyHostToDevice, cs));
        CK(cudaMemsetAsync(S->parts.p, 0, (np + P.n_extra) * sizeof(Partial), cs));
        CK(cudaStreamSynchronize(cs));
        N = P.N;
    }
    cudaStream_t s = S->sm;
    CK(cudaEventRecord(S->ev_start, s));
    uint32_t launches = 0;
    if (np > 0) {
        const bool per_pair = ctx->cfg.precision == PHMM_PREC_FP64 && (ctx->cfg.flags & PHMM_F_LAUNCH_PER_PAIR);
        const bool use_graph = !(ctx->cfg.flags & PHMM_F_NO_GRAPH) && !per_pair;
        if (per_pair) {
            const BatchHeader* H = static_cast<const BatchHeader*>(S->hdr.p);
            launch_reset(H, ctx->sms * 4, s);
            launch_prep64_all(H, static_cast<const PhredTables*>(ctx->tables.p), ctx->sms * 4, s);
            CK(cudaEventRecord(S->ev_fwd0, s));
            for (uint32_t p = 0; p < np; ++p) launch_single64(H, ctx->pow64.p, p, s);
            CK(cudaEventRecord(S->ev_fwd1, s));
            launch_finalize64(H, ctx->sms * 4, s);
            CK(cudaEventRecord(S->ev_res0, s));
            CK(cudaEventRecord(S->ev_res1, s));
            CK(cudaGetLastError());
            launches = np + 3;
        } else if (use_graph) {
            const int key = P.long_kind * 100000 + ctx->cfg.precision * 10000 + P.scal_id * 100 + (P.pack_id + 1);
            if (!S->gexec || S->g_key != key) {
                if (S->gexec) cudaGraphExecDestroy(S->gexec);
                S->gexec = nullptr;
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                const int rc = launch_sequence(ctx, *S, P.scal_id, P.pack_id, P.long_kind, true);
                cudaError_t e2 = cudaStreamEndCapture(s, &g);
                if (rc != PHMM_OK || e2 != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    ctx->dead = true;
                    return PHMM_ECUDA;
                }
                cudaError_t e3 = cudaGraphInstantiate(&S->gexec, g, 0);
                cudaGraphDestroy(g);
                CK(e3);
                S->g_key = key;
            }
            CK(cudaGraphLaunch(S->gexec, s));
            launches = (uint32_t)kernels_per_launch(ctx->cfg.precision, P.NP, P.scal_id);
        } else {
            const int rc = launch_sequence(ctx, *S, P.scal_id, P.pack_id, P.long_kind, false);
            if (rc != PHMM_OK) return rc;
            launches = (uint32_t)kernels_per_launch(ctx->cfg.precision, P.NP, P.scal_id);
        }
        // outputs
        if (b->outputs_on_device) {
            CK(cudaMemcpyAsync(b->out_log10, S->out.p, np * 8ull, cudaMemcpyDeviceToDevice, s));
            if (b->out_flags) CK(cudaMemcpyAsync(b->out_flags, S->oflags.p, np, cudaMemcpyDeviceToDevice, s));
        } else {
            CK(cudaMemcpyAsync(S->h_out.p, S->out.p, np * 8ull, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(S->h_oflags.p, S->oflags.p, np, cudaMemcpyDeviceToHost, s));
        }
        CK(cudaMemcpyAsync(S->h_small.p, S->small.p, 64, cudaMemcpyDeviceToHost, s));
    } else {
        memset(S->h_small.p, 0, 64);
        CK(cudaEventRecord(S->ev_fwd0, s));
        CK(cudaEventRecord(S->ev_fwd1, s));
        CK(cudaEventRecord(S->ev_res0, s));
        CK(cudaEventRecord(S->ev_res1, s));
    }
    CK(cudaEventRecord(S->ev_end, s));
    // later work on the caller's stream sees the outputs
    CK(cudaStreamWaitEvent(ctx->stream, S->ev_end, 0));
    S->foot = foot;
    ctx->inflight_foot += foot;
    S->ticket = ++ctx->next_ticket;
    S->state = 1;
    S->user_out = b->out_log10;
    S->user_flags = b->out_flags;
    S->out_on_dev = b->outputs_on_device != 0;
    S->n_pairs = np;
    S->has_stats = false;
    memset(&S->st, 0, sizeof(S->st));
    S->st.cells = cells;
    S->st.n_pairs = np;
    S->st.n_long = P.n_long;
    S->st.cols_per_lane = (uint32_t)(P.NP > 0 ? P.NP : N);
    S->st.kernel_launches = launches;
    {
        const bool f32 = ctx->cfg.precision != PHMM_PREC_FP64;
        // FP64: the forward variant (0: N 8 in 16-warp CTAs, 1: N 16 in 8-warp CTAs)
        S->st.short_kernel = f32 ? (!P.witems.empty() ? P.scal_id : -1) : P.scal_id;
        S->st.packed_kernel = f32 && !P.witems2.empty() ? P.pack_id : -1;
        S->st.long_kernel = f32 && !P.citems.empty() ? P.long_kind : -1;
        const bool branched = f32 || f64_pipelined(P.scal_id);  // the pipelined FP64 variants have two branches
        for (int q = 0; q < 3; ++q) S->st.cells_branch[q] = branched ? P.cells_br[q] : (q == 0 ? cells : 0);
    }
    S->host_status = P.n_too_long ? PHMM_EINVAL : PHMM_OK;
    S->plan_valid = true;
    S->plan_hash = hsh;
    S->plan_np = np;
    S->st.ms_host = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0).count();
    if (getenv("PHMM_DEBUG"))
        fprintf(stderr, "phmm submit: plan %s %.1f ms, host total %.1f ms\n", reuse ? "reused" : "built",
                std::chrono::duration<double, std::milli>(th_plan - th0).count(), S->st.ms_host);
    *ticket = S->ticket;
    return PHMM_OK;
}

int phmm_batch_footprint(phmm_ctx* ctx, const phmm_batch* b, uint64_t* bytes) {
    if (!ctx || !b || !bytes || b->inputs_on_device) return PHMM_EINVAL;
    *bytes = 0;
    const uint32_t nr = b->n_reads, nh = b->n_haps, np = b->n_pairs;
    if (np == 0) return PHMM_OK;
    if (!b->read_off || !b->hap_off || !b->pair_read || !b->pair_hap || nr == 0 || nh == 0) return PHMM_EINVAL;
    const uint64_t *roff = b->read_off, *hoff = b->hap_off;
    if (roff[0] != 0 || hoff[0] != 0) return PHMM_EINVAL;
    for (uint32_t r = 0; r < nr; ++r)
        if (roff[r + 1] <= roff[r] || roff[r + 1] - roff[r] > 0xffffffull) return PHMM_EINVAL;
    for (uint32_t h = 0; h < nh; ++h)
        if (hoff[h + 1] <= hoff[h] || hoff[h + 1] - hoff[h] > 0xffffffull) return PHMM_EINVAL;
    const int prec = ctx->cfg.precision;
    const bool need64 = prec != PHMM_PREC_FP32_ONLY;
    const uint64_t nbases = roff[nr], nhb = hoff[nh];
    const uint64_t seg = 32ull * (prec == PHMM_PREC_FP64 ? kN64 : kNLong32);
    uint64_t f = nbases * 5 + nhb + (nr + 1) * 8ull + (nh + 1) * 8ull + np * 8ull;
    f += nbases * ((prec != PHMM_PREC_FP64 ? sizeof(Rec32) + sizeof(Rec32J) : sizeof(Rec64J)) +
                   (need64 ? sizeof(Rec64) : 0));
    f += (uint64_t)np * (sizeof(PairDesc) + sizeof(Partial) + 8 + 1 + 4 + sizeof(Team) + 2 * sizeof(WarpItem) +
                         sizeof(CtaPair) + sizeof(CtaItem));
    uint64_t lmax = 0;
    for (uint32_t p = 0; p < np; ++p) {
        if (b->pair_read[p] >= nr || b->pair_hap[p] >= nh) return PHMM_EINVAL;
        const uint64_t l = roff[b->pair_read[p] + 1] - roff[b->pair_read[p]];
        const uint64_t k = hoff[b->pair_hap[p] + 1] - hoff[b->pair_hap[p]];
        lmax = std::max(lmax, l);
        const uint64_t Wt = (k + seg - 1) / seg;
        // the narrowest CTA strips of any FP32 multi-warp kind bound the boundary words
        const uint64_t cw = prec == PHMM_PREC_FP64 ? (uint64_t)kCtaWarps : (uint64_t)kLongCW[4];
        if (Wt > cw) {  // strips of a very wide pair
            const uint64_t S = (Wt + cw - 1) / cw;
            f += (S - 1) * (l * (prec == PHMM_PREC_FP64 ? 8 : 4) * 8 + sizeof(Partial) + sizeof(CtaPair) + sizeof(CtaItem));
        }
    }
    if (need64) f += (uint64_t)ctx->sms * ctx->occ64 * 2 * lmax * 8 * 8 + 16;
    if (prec != PHMM_PREC_FP64)  // serial multi-warp kind: two boundaries per resident warp
        f += (uint64_t)ctx->sms * ctx->occ_longk[3] * (kSerialThreads / 32) * 2 * lmax * sizeof(float4);
    *bytes = f;
    return PHMM_OK;
}

int phmm_poll(phmm_ctx* ctx, uint64_t ticket, int timeout_ms) {
    if (!ctx) return PHMM_EINVAL;
    Slot* S = nullptr;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        for (auto& s : ctx->slots)
            if (s.state == 1 && s.ticket == ticket) S = &s;
        if (!S) return PHMM_ENOTFOUND;
    }
    cudaSetDevice(ctx->dev);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(S->ev_end);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) {
            ctx->dead = true;
            return PHMM_ECUDA;
        }
        if (timeout_ms == 0) return PHMM_PENDING;
        if (timeout_ms > 0) {
            const double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_ms) return PHMM_PENDING;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!S->out_on_dev && S->n_pairs > 0) {
        memcpy(S->user_out, S->h_out.p, S->n_pairs * 8ull);
        if (S->user_flags) memcpy(S->user_flags, S->h_oflags.p, S->n_pairs);
    }
    const uint32_t* sm = static_cast<const uint32_t*>(S->h_small.p);
    S->st.n_rescued = sm[2];
    S->st.status_bits = sm[8];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, S->ev_start, S->ev_end);
    S->st.ms_total = ms;
    ms = 0.f;
    cudaEventElapsedTime(&ms, S->ev_fwd0, S->ev_fwd1);
    S->st.ms_forward = ms;
    ms = 0.f;
    cudaEventElapsedTime(&ms, S->ev_res0, S->ev_res1);
    S->st.ms_rescue = ms;
    for (int q = 0; q < 3; ++q) {
        ms = 0.f;
        if (S->br_timed && (S->br_mask >> q & 1u)) cudaEventElapsedTime(&ms, S->ev_br[2 * q], S->ev_br[2 * q + 1]);
        S->st.ms_branch[q] = ms;
    }
    if (!S->br_timed) S->st.ms_branch[0] = S->st.ms_forward;  // FP64: one forward kernel
    ctx->last_stats = S->st;
    ctx->last_retired = S->ticket;
    ctx->inflight_foot -= S->foot;
    S->foot = 0;
    S->state = 0;
    int rc = S->host_status;
    if (sm[8] & ST_TIMEOUT) rc = PHMM_ETIMEOUT;
    else if (sm[8] & (ST_BAD_INPUT | ST_TOO_LONG)) rc = PHMM_EINVAL;
    return rc;
}

int phmm_get_stats(phmm_ctx* ctx, uint64_t ticket, phmm_stats* out) {
    if (!ctx || !out) return PHMM_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ticket == ctx->last_retired) {
        *out = ctx->last_stats;
        return PHMM_OK;
    }
    for (auto& s : ctx->slots)
        if (s.state == 1 && s.ticket == ticket) {
            *out = s.st;
            return PHMM_PENDING;
        }
    return PHMM_ENOTFOUND;
}

int phmm_plan_check(const uint32_t* l, const uint32_t* k, const uint32_t* pair_read, uint32_t n,
                    int precision, int scal_id, int pack_id, int long_kind, uint64_t* stats) {
    if (!l || !k || !pair_read || !stats) return PHMM_EINVAL;
    if (precision < 0 || precision > 2) return PHMM_EINVAL;
    for (int q = 0; q < 8; ++q) stats[q] = 0;
    Plan P;
    int CW = kCtaWarps, Nl = kN64, kw = 8;
    if (precision == PHMM_PREC_FP64) {
        if (scal_id < 0 || scal_id >= kNumF64) return PHMM_EINVAL;  // the FP64 variant
        make_plan64(l, k, pair_read, n, scal_id, P);
        CW = kF64CW[scal_id];
        Nl = kF64N[scal_id];
    } else {
        if (scal_id < 0 || scal_id >= kNumScalar || pack_id < -1 || pack_id >= kNumPacked || long_kind < 0 ||
            long_kind >= kNumLong)
            return PHMM_EINVAL;
        make_plan_id(l, k, pair_read, n, scal_id, pack_id, long_kind, P);
        CW = kLongCW[long_kind];
        Nl = kLongN[long_kind];
        kw = 4;
    }
    const uint64_t seg = 32ull * (uint64_t)Nl;
    auto fail = [&](uint64_t code) {
        stats[7] = code;
        return PHMM_EINVAL;
    };
    std::vector<uint32_t> seen(n, 0);
    // teams: inside their warp, disjoint, wide enough, packed pairs share a read
    auto check_items = [&](const std::vector<WarpItem>& items, bool packed) -> int {
        for (const WarpItem& w : items) {
            uint64_t used = 0;
            for (uint32_t t = 0; t < w.n_teams; ++t) {
                if (w.first_team + t >= P.teams.size()) return 1;
                const Team& tm = P.teams[w.first_team + t];
                if (tm.size == 0 || tm.base + tm.size > 32) return 2;
                const uint64_t bits = ((tm.size == 32 ? ~0ull : ((1ull << tm.size) - 1)) << tm.base) & 0xffffffffull;
                if (used & bits) return 3;
                used |= bits;
                const int Nw = packed ? P.NP : P.N;
                if (tm.pair >= n) return 4;
                if ((uint64_t)tm.size * Nw < k[tm.pair]) return 5;
                seen[tm.pair]++;
                if (tm.pair2 != kNoPair) {
                    if (!packed || tm.pair2 >= n) return 6;
                    if (pair_read[tm.pair2] != pair_read[tm.pair]) return 7;
                    if ((uint64_t)tm.size * Nw < k[tm.pair2]) return 5;
                    seen[tm.pair2]++;
                }
            }
        }
        return 0;
    };
    if (int e = check_items(P.witems, false)) return fail(e);
    if (int e = check_items(P.witems2, true)) return fail(e);
    // CTA items: warp ranges fit and are disjoint; strips tile their pair in item order
    struct StripSeen {
        uint32_t nstrip = 0, count = 0, extra_base = 0;
        std::vector<int64_t> col0, width, item, w0;
        std::vector<uint64_t> bin, bout, pad;
    };
    std::map<uint32_t, StripSeen> strips;
    std::vector<std::pair<uint64_t, uint64_t>> bnd_ranges, extra_ranges;
    const bool serial = precision != PHMM_PREC_FP64 && kLongSerial[long_kind];
    // wave kind: one strip per item on one warp; boundaries are float4 rows of wbnd and
    // each strip's progress is boundary word `pad` (consecutive within a pair)
    const bool wave = precision != PHMM_PREC_FP64 && kLongWave[long_kind];
    std::vector<std::pair<uint64_t, uint64_t>> prog_ranges;
    for (size_t it = 0; it < P.citems.size(); ++it) {
        const CtaItem& ci = P.citems[it];
        uint32_t used = 0;
        for (uint32_t q = 0; q < ci.n; ++q) {
            if (ci.first + q >= P.cpairs.size()) return fail(10);
            const CtaPair& cp = P.cpairs[ci.first + q];
            if (cp.W == 0 || cp.w0 + cp.W > CW) return fail(11);
            const uint32_t bits = ((cp.W == 32 ? ~0u : ((1u << cp.W) - 1)) << cp.w0);
            if (used & bits) return fail(12);
            used |= bits;
            if (cp.pair >= n) return fail(13);
            const uint64_t Wt = (k[cp.pair] + seg - 1) / seg;
            if (serial) {
                // one pair per item, all its strips on one warp; strips 1.. leave their
                // partials at extra_base + s - 1
                if (ci.n != 1 || cp.W != 1 || cp.w0 != 0 || cp.col0 != 0 || cp.bnd_in != kNoBnd ||
                    cp.bnd_out != kNoBnd)
                    return fail(16);
                if (cp.nstrip != Wt) return fail(17);
                if (l[cp.pair] > P.serial_rows) return fail(18);
                if (cp.nstrip > 1) {
                    if (cp.extra_base < n || cp.extra_base + cp.nstrip - 1 > n + P.n_extra) return fail(27);
                    extra_ranges.push_back({cp.extra_base, cp.extra_base + cp.nstrip - 1});
                    stats[5]++;
                }
                seen[cp.pair]++;
                continue;
            }
            if (cp.nstrip <= 1) {
                if (cp.W != Wt || cp.col0 != 0 || cp.bnd_in != kNoBnd || cp.bnd_out != kNoBnd) return fail(14);
                seen[cp.pair]++;
                continue;
            }
            StripSeen& sv = strips[cp.pair];
            if (sv.count == 0) {
                sv.nstrip = cp.nstrip;
                sv.extra_base = cp.extra_base;
                sv.col0.assign(cp.nstrip, -1);
                sv.width.assign(cp.nstrip, -1);
                sv.item.assign(cp.nstrip, -1);
                sv.w0.assign(cp.nstrip, -1);
                sv.bin.assign(cp.nstrip, 0);
                sv.bout.assign(cp.nstrip, 0);
                sv.pad.assign(cp.nstrip, 0);
            }
            if (wave && (ci.n != 1 || cp.W != 1 || cp.w0 != 0)) return fail(31);
            if (cp.nstrip != sv.nstrip || cp.extra_base != sv.extra_base || cp.strip >= sv.nstrip ||
                sv.item[cp.strip] >= 0)
                return fail(15);
            sv.col0[cp.strip] = cp.col0;
            sv.width[cp.strip] = cp.W;
            sv.item[cp.strip] = (int64_t)it;
            sv.w0[cp.strip] = cp.w0;
            sv.bin[cp.strip] = cp.bnd_in;
            sv.bout[cp.strip] = cp.bnd_out;
            sv.pad[cp.strip] = cp.pad;
            sv.count++;
        }
    }
    for (auto& kv : strips) {
        const uint32_t p = kv.first;
        StripSeen& sv = kv.second;
        if (sv.count != sv.nstrip) return fail(20);
        int64_t col = 0, warps = 0;
        for (uint32_t st = 0; st < sv.nstrip; ++st) {
            if (sv.col0[st] != col) return fail(21);
            col += sv.width[st] * (int64_t)seg;
            warps += sv.width[st];
            if (st > 0 && sv.item[st] < sv.item[st - 1]) return fail(22);  // never before its left strip
            if ((st == 0) != (sv.bin[st] == kNoBnd)) return fail(23);
            if ((st + 1 == sv.nstrip) != (sv.bout[st] == kNoBnd)) return fail(23);
            if (st > 0) {
                const bool din = is_dsmem_bnd(sv.bin[st]);
                if (din != is_dsmem_bnd(sv.bout[st - 1])) return fail(28);
                if (din) {
                    // distributed shared memory: neighbouring CTAs of one cluster group, and
                    // the left strip names the receiving strip's first warp
                    if (long_kind != 5 || precision == PHMM_PREC_FP64) return fail(28);
                    if (sv.item[st] != sv.item[st - 1] + 1 || sv.item[st] % kClusterCtas == 0) return fail(29);
                    if ((int64_t)(sv.bout[st - 1] & 0xffu) != sv.w0[st]) return fail(29);
                } else if (sv.bin[st] != sv.bout[st - 1]) {
                    return fail(24);
                }
            }
            if (wave) {
                if (sv.pad[st] != sv.pad[0] + st) return fail(32);
                if (st + 1 < sv.nstrip) {
                    const uint64_t a = sv.bout[st], b = a + (uint64_t)l[p];
                    if (b > P.wave_rows) return fail(25);
                    bnd_ranges.push_back({a, b});
                }
                continue;
            }
            if (st + 1 < sv.nstrip && !is_dsmem_bnd(sv.bout[st])) {
                const uint64_t a = sv.bout[st], b = a + (uint64_t)l[p] * kw;
                if (b > P.bnd_words) return fail(25);
                bnd_ranges.push_back({a, b});
            }
        }
        if ((uint64_t)warps != (k[p] + seg - 1) / seg) return fail(26);
        if (wave) {
            if (sv.pad[0] + sv.nstrip > P.bnd_words) return fail(32);
            prog_ranges.push_back({sv.pad[0], sv.pad[0] + sv.nstrip});
        }
        if (sv.extra_base < n || sv.extra_base + sv.nstrip - 1 > n + P.n_extra) return fail(27);
        extra_ranges.push_back({sv.extra_base, sv.extra_base + sv.nstrip - 1});
        seen[p]++;
        stats[5]++;
    }
    auto disjoint = [](std::vector<std::pair<uint64_t, uint64_t>>& r) {
        std::sort(r.begin(), r.end());
        for (size_t q = 1; q < r.size(); ++q)
            if (r[q].first < r[q - 1].second) return false;
        return true;
    };
    if (!disjoint(bnd_ranges)) return fail(28);
    if (!disjoint(prog_ranges)) return fail(32);
    if (!disjoint(extra_ranges)) return fail(29);
    for (uint32_t p = 0; p < n; ++p)
        if (seen[p] != 1) return fail(30);
    stats[0] = P.teams.size();
    stats[1] = P.witems.size();
    stats[2] = P.witems2.size();
    stats[3] = P.citems.size();
    stats[4] = P.cpairs.size();
    stats[6] = P.n_too_long;
    return PHMM_OK;
}

int phmm_wait_test(phmm_ctx* ctx) {
    if (!ctx) return PHMM_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->dead) return PHMM_ECUDA;
    cudaSetDevice(ctx->dev);
    DevBuf buf;
    CK(ensure(buf, 64));
    CK(cudaMemsetAsync(buf.p, 0, 64, ctx->stream));
    uint32_t* status = static_cast<uint32_t*>(buf.p) + 12;  // word after the 4 boundary words
    launch_wait_test(buf.p, status, ctx->stream);
    CK(cudaGetLastError());
    uint32_t st = 0;
    CK(cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    release(buf);
    return (st & ST_TIMEOUT) ? PHMM_ETIMEOUT : PHMM_OK;
}

int phmm_scan_test(phmm_ctx* ctx, const float* y, float* z, int n, float a) {
    if (!ctx || !y || !z || n < 1 || n > 1024 || !(a >= 0.0f) || !(a <= 1.0f)) return PHMM_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaSetDevice(ctx->dev);
    PowRow<float> row{};
    const double la = a > 0.0f ? std::log10((double)a) : -1e9;
    for (int s = 0; s < 5; ++s) {
        const double m = 32.0 * (1 << s);
        const double lg = la * m;
        if (lg >= std::log10((double)std::numeric_limits<float>::min())) {
            row.sp1[s] = (float)std::pow(10.0, lg);
            row.sp2[s] = 1.0f;
        } else {
            row.sp1[s] = row.sp2[s] = (float)std::pow(10.0, lg / 2.0);
        }
    }
    row.pad1 = a;
    CK(ensure(ctx->scan_row, sizeof(row)));
    CK(cudaMemcpyAsync(ctx->scan_row.p, &row, sizeof(row), cudaMemcpyHostToDevice, ctx->stream));
    launch_scan_test(y, z, n, ctx->scan_row.p, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return PHMM_OK;
}

}  // extern "C"
