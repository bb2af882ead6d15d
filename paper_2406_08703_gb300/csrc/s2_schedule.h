// Work split of the intensity contraction (stage 2: I += w |A(l) . T1t[b]^T|^2
// summed over the wavelengths l of one output tile), host side.
//
// A segment is one 128x128 output tile of one (slot, source, exposure); it has
// n_lambda jobs, one per wavelength, whose |E|^2 terms add up in the registers
// of the CTA that runs them.  A piece is a run of consecutive wavelengths of one
// segment given to one CTA; it ends with a store of its partial sum into one of
// `planes` partial-intensity planes, which the binning pass adds up.
//
// The split keeps the CTAs that run at the same time on the same wavelength,
// so the A(l) and T1t rows one wavelength needs are read from HBM once and
// shared through L2 by every tile that uses them:
//  * whole segments, one per CTA per round, while every CTA gets one;
//  * the rs < CTAs segments left: CTA c < rs takes wavelengths [0, Lm) of
//    segment c (Lm = ceil(rs n_lambda / CTAs)), all in step; the remaining
//    wavelengths [Lm, n_lambda) of those segments are cut into equal contiguous
//    runs for the other CTAs.  The last piece of a segment marks the first plane it left
//    unwritten, and that CTA clears the planes from there on, so every plane
//    the binning pass reads holds a partial sum or zero.
#pragma once
#include <algorithm>
#include <string>
#include <vector>

namespace dlx {

struct S2Piece {
    int seg, l0, l1;
    int pz;  // plane | (first plane to clear << 16); kS2None: nothing to clear
};
constexpr int kS2None = 0x7fff;

// Builds the pieces of each CTA: CTA c runs pcs[off[c] .. off[c+1]).  Returns
// the number of planes the split writes.
inline int s2_split(int nseg, int nl, int nct, std::vector<int> &off, std::vector<S2Piece> &pcs) {
    off.assign(nct + 1, 0);
    pcs.clear();
    if (nseg <= 0 || nl <= 0 || nct <= 0) return 1;
    std::vector<std::vector<S2Piece>> per(nct);
    // whole segments while every CTA gets one
    const int rounds = nseg / nct, s0 = rounds * nct, rs = nseg - s0;
    for (int k = 0; k < rounds; ++k)
        for (int c = 0; c < nct; ++c) per[c].push_back({k * nct + c, 0, nl, 0 | (1 << 16)});
    int planes = 1;
    if (rs > 0) {
        // the rs < nct remaining segments: heads in step, tails cut evenly
        const long jobs = (long)rs * nl;
        const int Lm = (int)std::min<long>(nl, (jobs + nct - 1) / nct);
        const int tl = nl - Lm, nt = nct - rs;
        const long T = (long)rs * tl;  // tail jobs: segment-major, wavelength fastest
        std::vector<int> npieces(rs, 0);
        std::vector<std::pair<int, int>> last(rs, {-1, -1});  // (cta, index) of each segment's last piece
        for (int c = 0; c < rs; ++c) {
            per[c].push_back({s0 + c, 0, Lm, 0 | (kS2None << 16)});
            last[c] = {c, (int)per[c].size() - 1};
        }
        for (int i = 0; i < nt && T > 0; ++i) {
            const int c = rs + i;
            long t = T * i / nt;
            const long t1 = T * (i + 1) / nt;
            while (t < t1) {
                const int sg = (int)(t / tl), l = Lm + (int)(t % tl);
                const int l1 = (int)std::min<long>(nl, l + (t1 - t));
                const int plane = 1 + npieces[sg]++;
                per[c].push_back({s0 + sg, l, l1, plane | (kS2None << 16)});
                last[sg] = {c, (int)per[c].size() - 1};
                t += l1 - l;
            }
        }
        for (int sg = 0; sg < rs; ++sg) {
            const int used = 1 + npieces[sg];
            planes = std::max(planes, used);
            S2Piece &pc = per[last[sg].first][last[sg].second];
            pc.pz = (pc.pz & 0xffff) | (used << 16);
        }
    }
    for (int c = 0; c < nct; ++c) {
        off[c] = (int)pcs.size();
        pcs.insert(pcs.end(), per[c].begin(), per[c].end());
    }
    off[nct] = (int)pcs.size();
    return planes;
}

// The split for up to `max_cta` CTAs with at most kS2MaxPlanes planes: when a
// short tail would be cut into more pieces than that, fewer CTAs are used.
// Returns the planes written; `nct` receives the CTA count.
constexpr int kS2MaxPlanes = 16;
inline int s2_schedule(int nseg, int nl, int max_cta, int &nct, std::vector<int> &off, std::vector<S2Piece> &pcs) {
    nct = (int)std::max<long>(1, std::min<long>(max_cta, (long)nseg * nl));
    for (;;) {
        const int planes = s2_split(nseg, nl, nct, off, pcs);
        if (planes <= kS2MaxPlanes || nct == 1) return planes;
        nct = std::max(1, nct * 3 / 4);
    }
}

// Checks a split: every (segment, wavelength) job exactly once; per segment
// the written planes are 0 .. used-1, each once, and exactly one piece clears
// from `used` on.  Returns false with a reason otherwise.
inline bool s2_check(int nseg, int nl, int nct, const std::vector<int> &off, const std::vector<S2Piece> &pcs,
                     int planes, std::string *why) {
    std::vector<unsigned char> job((size_t)nseg * nl, 0);
    std::vector<int> written((size_t)nseg * planes, 0), clears(nseg, 0), used(nseg, 0);
    if ((int)off.size() != nct + 1 || off[0] != 0 || off[nct] != (int)pcs.size()) {
        *why = "stage-2 split: bad offsets";
        return false;
    }
    for (int c = 0; c < nct; ++c) {
        if (off[c + 1] < off[c]) {
            *why = "stage-2 split: offsets not ascending";
            return false;
        }
    }
    for (const S2Piece &pc : pcs) {
        const int plane = pc.pz & 0xffff, zf = pc.pz >> 16;
        if (pc.seg < 0 || pc.seg >= nseg || pc.l0 < 0 || pc.l1 > nl || pc.l0 >= pc.l1 || plane >= planes) {
            *why = "stage-2 split: piece out of range";
            return false;
        }
        for (int l = pc.l0; l < pc.l1; ++l) job[(size_t)pc.seg * nl + l]++;
        written[(size_t)pc.seg * planes + plane]++;
        if (zf != kS2None) {
            clears[pc.seg]++;
            used[pc.seg] = zf;
        }
    }
    for (size_t i = 0; i < job.size(); ++i)
        if (job[i] != 1) {
            *why = "stage-2 split: a job is not covered exactly once";
            return false;
        }
    for (int s = 0; s < nseg; ++s) {
        if (clears[s] != 1 || used[s] < 1 || used[s] > planes) {
            *why = "stage-2 split: a segment lacks its single clearing piece";
            return false;
        }
        for (int q = 0; q < planes; ++q)
            if (written[(size_t)s * planes + q] != (q < used[s] ? 1 : 0)) {
                *why = "stage-2 split: planes of a segment not written exactly once";
                return false;
            }
    }
    return true;
}

}  // namespace dlx
