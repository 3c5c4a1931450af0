// quad_tiling.h -- host-side tables of the shared-partial-sum dedispersion
// kernel (dedisp_quad_kernel, dedisp.cu).
//
// Channels are taken four at a time (a quad; the last one may be shorter).
// Within a DM tile, trial j sees quad q's channels at delays
// o_k(j) = delay(4q + k, j); the vector v(j) = (o_1 - o_0, o_2 - o_0, o_3 - o_0)
// repeats across neighbouring trials, so the quad's sum for trial j,
//   sum_k x_{4q+k}[t + o_k(j)] = P_v[t + o_0(j)],
//   P_v[u] = sum_k x_{4q+k}[u + v_k],
// is one entry of a partial-sum row P_v shared by every trial with that
// vector (a pattern).  The kernel's builder warps form each pattern's row in
// shared memory (16-bit sums, at most 4 * 255) over the samples its trials
// need, and its consumer warps add, per trial, the 16-bit row entries at the
// trial's own offset.  The sums are exactly those of direct dedispersion.
//
// Per stage (a run of consecutive quads, at most 256 channels) the slot in
// shared memory holds, in this order and at byte offsets the plan fixes:
//   ChanDesc [nchan]                            (copied)
//   QPattern [npat], then the consumer table    (copied, the stage's addr words)
//     consumer table: [quad pair][BD] x {addr q0, addr q1, sel q0, sel q1}
//   byte rows of the stage's channels           (copied, 16-byte aligned)
//   pattern rows                                (built by the kernel)
#pragma once

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include "hp_internal.h"

namespace hp {

// One pattern of a stage: built into `dst` (byte offset in the slot, 8-byte
// aligned) as ngroups groups of four 16-bit samples; channel k of the quad is
// read from byte src[k] of the slot (4-byte aligned) and aligned by PRMT
// selector sel[k].  48 bytes.
struct QPattern {
    uint32_t dst;
    uint32_t ngroups;
    uint32_t nk;
    uint32_t pad_;
    uint32_t src[4];
    uint32_t sel[4];
};
static_assert(sizeof(QPattern) == 48, "QPattern layout");

constexpr int kQuadGroupsPerLane = 7;   // builder lanes take 7 consecutive 4-sample groups (odd: no bank conflicts)

inline uint32_t q_align(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// Stages, channel descriptors and tables of one DM tile of nd trials (delay(j, c)
// of trial j, channel c) for a quad configuration C; appends to T.  Returns
// HP_OK or HP_ERR_INVALID_ARG when one quad does not fit a slot.
template <class Delay>
int append_tile_quad(const Delay& delay, int nd, int nch, int32_t d0, const DedispConfig& C,
                     DedispTiling* T) {
    const int BD = C.BD(), BT = C.BT();
    const uint32_t budget = (uint32_t)C.stage_bytes;
    const int nq = (nch + 3) / 4;
    struct Pat {
        int32_t lo, hi;            // sample range of the row, relative to the tile start
        int32_t v[4];              // delays of the quad's channels relative to channel 0
        std::vector<int> trials;
    };
    struct Quad {
        int c0, nk;
        int32_t base[4];           // staged row start of each channel (16-byte aligned)
        uint32_t rowbytes[4];
        std::vector<Pat> pats;
        std::vector<int> pat_of;   // [BD] pattern of trial j (j >= nd: trial 0's)
        uint32_t pat_words_total;  // 32-bit words of all pattern rows
    };
    std::vector<Quad> quads(nq);
    for (int q = 0; q < nq; ++q) {
        Quad& Q = quads[q];
        Q.c0 = 4 * q;
        Q.nk = std::min(4, nch - Q.c0);
        std::map<std::vector<int32_t>, int> index;
        Q.pat_of.assign(BD, 0);
        for (int j = 0; j < nd; ++j) {
            const int32_t o0 = delay(j, Q.c0);
            std::vector<int32_t> v(4, 0);
            for (int k = 1; k < Q.nk; ++k) v[k] = delay(j, Q.c0 + k) - o0;
            auto it = index.find(v);
            int p;
            if (it == index.end()) {
                p = (int)Q.pats.size();
                index.emplace(v, p);
                Pat P;
                P.lo = o0;
                P.hi = o0 + BT;
                for (int k = 0; k < 4; ++k) P.v[k] = v[k];
                Q.pats.push_back(P);
            } else {
                p = it->second;
            }
            Pat& P = Q.pats[p];
            P.lo = std::min(P.lo, o0);
            P.hi = std::max(P.hi, o0 + BT);
            P.trials.push_back(j);
            Q.pat_of[j] = p;
        }
        // pattern rows: every sample the builders write (whole groups, rounded to
        // a lane's 7 groups) and every word a consumer lane reads (the trial's
        // first word + BT/2, one word past its last sample)
        Q.pat_words_total = 0;
        for (Pat& P : Q.pats) {
            const uint32_t ng = (uint32_t)(P.hi - P.lo + 3) / 4;
            uint32_t words = q_align(ng, kQuadGroupsPerLane) * 2;
            for (int j : P.trials) {
                const uint32_t s = (uint32_t)(delay(j, Q.c0) - P.lo);
                words = std::max(words, (s >> 1) + (uint32_t)BT / 2 + 1);
            }
            Q.pat_words_total += q_align(words, 2);
        }
        // staged rows: from the channel's smallest delay rounded down to 16 bytes,
        // to the last word the builders read (7 groups per lane, one extra word)
        for (int k = 0; k < Q.nk; ++k) {
            const int c = Q.c0 + k;
            int32_t lo = delay(0, c);
            for (int j = 1; j < nd; ++j) lo = std::min(lo, delay(j, c));
            Q.base[k] = lo & ~15;
            uint32_t end = 0;
            for (const Pat& P : Q.pats) {
                const uint32_t ng = (uint32_t)(P.hi - P.lo + 3) / 4;
                const uint32_t rel = (uint32_t)(P.lo + P.v[k] - Q.base[k]);
                end = std::max(end, (rel & ~3u) + 4 * q_align(ng, kQuadGroupsPerLane) + 4);
            }
            Q.rowbytes[k] = q_align(end, 16);
        }
    }

    TileDesc td;
    td.d0 = d0;
    td.nd = nd;
    td.stage_begin = (int32_t)T->stages.size();
    td.nstages = 0;
    auto stage_bytes = [&](int q_begin, int q_end, uint32_t* tab_bytes) {
        int nchan = 0, npat = 0;
        uint32_t rows = 0, pat = 0;
        for (int q = q_begin; q < q_end; ++q) {
            nchan += quads[q].nk;
            npat += (int)quads[q].pats.size();
            for (int k = 0; k < quads[q].nk; ++k) rows += quads[q].rowbytes[k];
            pat += 4 * quads[q].pat_words_total;
        }
        const int npairs = (q_end - q_begin + 1) / 2;
        const uint32_t tb = (uint32_t)npat * sizeof(QPattern) + (uint32_t)npairs * BD * 16;
        if (tab_bytes) *tab_bytes = tb;
        return q_align((uint32_t)nchan * sizeof(ChanDesc), 16) + q_align(tb, 16) + rows +
               q_align(pat, 16);
    };
    int q = 0;
    while (q < nq) {
        int q_end = q + 1;
        if (stage_bytes(q, q_end, nullptr) > budget) return HP_ERR_INVALID_ARG;
        int nchan = quads[q].nk;
        while (q_end < nq && nchan + quads[q_end].nk <= kStageMaxChans &&
               stage_bytes(q, q_end + 1, nullptr) <= budget) {
            nchan += quads[q_end].nk;
            ++q_end;
        }
        uint32_t tab_bytes = 0;
        stage_bytes(q, q_end, &tab_bytes);
        int npat = 0;
        for (int i = q; i < q_end; ++i) npat += (int)quads[i].pats.size();
        const int nqs = q_end - q;
        StageDesc sd{};
        sd.chan_begin = (uint32_t)T->chans.size();
        sd.nchan = (uint32_t)nchan;
        sd.addr_off = q_align((uint32_t)nchan * sizeof(ChanDesc), 16);
        sd.addr_begin = (uint32_t)T->addr.size();
        sd.addr_bytes = tab_bytes;
        sd.npat = (uint32_t)npat;
        sd.ctab_off = sd.addr_off + (uint32_t)npat * sizeof(QPattern);
        uint32_t off = sd.addr_off + q_align(tab_bytes, 16);
        uint32_t tx = (uint32_t)(nchan * sizeof(ChanDesc)) + tab_bytes;
        // rows
        std::vector<std::array<uint32_t, 4>> rowoff(nqs);
        for (int i = 0; i < nqs; ++i) {
            const Quad& Q = quads[q + i];
            for (int k = 0; k < Q.nk; ++k) {
                ChanDesc cd;
                cd.c = (uint32_t)(Q.c0 + k);
                cd.goff = Q.base[k];
                cd.offB = off;
                cd.nwords = Q.rowbytes[k] / 4;
                T->chans.push_back(cd);
                rowoff[i][k] = off;
                off += Q.rowbytes[k];
                tx += Q.rowbytes[k];
                T->max_reach = std::max<int64_t>(T->max_reach, (int64_t)Q.base[k] + Q.rowbytes[k]);
            }
        }
        // pattern rows and the builder table
        std::vector<std::vector<uint32_t>> pdst(nqs);
        for (int i = 0; i < nqs; ++i) {
            const Quad& Q = quads[q + i];
            for (const Pat& P : Q.pats) {
                const uint32_t ng = (uint32_t)(P.hi - P.lo + 3) / 4;
                uint32_t words = q_align(ng, kQuadGroupsPerLane) * 2;
                for (int j : P.trials) {
                    const uint32_t s = (uint32_t)(delay(j, Q.c0) - P.lo);
                    words = std::max(words, (s >> 1) + (uint32_t)BT / 2 + 1);
                }
                pdst[i].push_back(off);
                QPattern e{};
                e.dst = off;
                e.ngroups = ng;
                e.nk = (uint32_t)Q.nk;
                for (int k = 0; k < 4; ++k) {
                    const int kk = k < Q.nk ? k : 0;
                    const uint32_t rel = (uint32_t)(P.lo + P.v[kk] - Q.base[kk]);
                    e.src[k] = rowoff[i][kk] + (rel & ~3u);
                    e.sel[k] = 0x3210u + 0x1111u * (rel & 3u);
                }
                const uint32_t* w = reinterpret_cast<const uint32_t*>(&e);
                T->addr.insert(T->addr.end(), w, w + sizeof(QPattern) / 4);
                off += 4 * q_align(words, 2);
            }
        }
        if (off > budget) return HP_ERR_INVALID_ARG;
        // consumer table: per quad pair and trial, the first word each quad's
        // pattern row is read from (byte offset in the slot) and the PRMT selector
        // that takes the trial's two samples from a word pair
        for (int pr = 0; pr < (nqs + 1) / 2; ++pr) {
            for (int j = 0; j < BD; ++j) {
                uint32_t a[2], sel[2];
                for (int e = 0; e < 2; ++e) {
                    const int i = 2 * pr + e < nqs ? 2 * pr + e : 2 * pr;
                    const Quad& Q = quads[q + i];
                    const int jj = j < nd ? j : 0;
                    const int p = Q.pat_of[jj];
                    const uint32_t s = (uint32_t)(delay(jj, Q.c0) - Q.pats[p].lo);
                    a[e] = pdst[i][p] + 4 * (s >> 1);
                    sel[e] = (s & 1u) ? 0x5432u : 0x3210u;
                }
                T->addr.push_back(a[0]);
                T->addr.push_back(a[1]);
                T->addr.push_back(sel[0]);
                T->addr.push_back(sel[1]);
            }
        }
        sd.tx_bytes = tx;
        T->stages.push_back(sd);
        td.nstages++;
        q = q_end;
    }
    T->tiles.push_back(td);
    return HP_OK;
}

}  // namespace hp
