// Host build of the kernel's own per-pixel scan (paper_2412_11639_gb300/csrc/spk_scan.cuh),
// driven word by word exactly as the CUDA kernel drives it: the first spike opens the
// stream, an all-ones word may be absorbed whole, every other spike goes through spike().
// It writes each pixel's stable sequences so that a test can compare them with the oracle
// on the CPU, and it checks the two properties the kernel's record ring relies on:
//   * a candidate arrives at most one place before its predecessor (the ring's single swap
//     restores time order), and
//   * no candidate arrives before a frontier() reported after an earlier word, and no two
//     cuts share a time (so a record at or before the frontier is final).
//
// usage: scan_host <stream.bin> <P> <T> <pitch> <order 1..5>[l] <out.bin>
// (1 FSR, 2 SSR: PixelScan; 3..5: the n-order tree TreeScan<n, 3> of the same header, its
// first three levels' node state indexed by constants; with the suffix l, TreeScan<n, 1>)
// stream.bin: uint8 [T][pitch], pixel p is bit p % 8 of byte p / 8 (the library's layout).
// out.bin: int32 counts[P], then for every pixel in order its sequences as int32 triples
// (t_start, t_end, n_intervals).  Exit status 0, or 3 if a property above failed.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <vector>

#include "../../paper_2412_11639_gb300/csrc/spk_scan.cuh"

namespace {

struct Cuts {
    std::vector<int> t, i;
    void cand(int tc, int ic) {
        t.push_back(tc);
        i.push_back(ic);
    }
    void put(bool emit, int tc, int ic) {
        if (emit) cand(tc, ic);
    }
};

template <int ORDER>
int run(const std::vector<uint8_t> &s, int64_t P, int T, int64_t pitch, FILE *out) {
    std::vector<int32_t> counts(P, 0), spans;
    int bad = 0;
    for (int64_t p = 0; p < P; ++p) {
        spk::PixelScan<ORDER> sc;
        sc.init();
        Cuts c;
        int t0 = -1, frontier = -1;  // latest frontier reported after a word
        size_t checked = 0;          // candidates already checked against a frontier
        for (int base = 0; base < T; base += 32) {
            uint32_t w = 0;
            for (int k = 0; k < 32 && base + k < T; ++k)
                w |= static_cast<uint32_t>((s[(base + k) * pitch + p / 8] >> (p % 8)) & 1) << k;
            if (sc.last_t < 0 && w) {
                t0 = base + __builtin_ctz(w);
                sc.first_spike(t0);
                w &= w - 1;
            }
            if (w == 0xffffffffu && sc.absorb_ones(base)) w = 0;
            while (w) {
                const int b = __builtin_ctz(w);
                w &= w - 1;
                sc.spike(base + b, c);
            }
            for (; checked < c.t.size(); ++checked)
                if (c.t[checked] < frontier) bad |= 2;
            if (sc.last_t >= 0) frontier = sc.frontier();
        }
        sc.finish(c);
        for (; checked < c.t.size(); ++checked)
            if (c.t[checked] < frontier) bad |= 2;
        // one adjacent swap per candidate, as the record ring does, then strictly increasing
        for (size_t j = 1; j < c.t.size(); ++j)
            if (c.t[j] < c.t[j - 1]) {
                std::swap(c.t[j], c.t[j - 1]);
                std::swap(c.i[j], c.i[j - 1]);
                if (j >= 2 && c.t[j - 1] <= c.t[j - 2]) bad |= 1;
            }
        for (size_t j = 1; j < c.t.size(); ++j)
            if (c.t[j] <= c.t[j - 1]) bad |= 1;
        int ct = t0, ci = -1;
        for (size_t j = 0; j < c.t.size(); ++j) {
            spans.push_back(ct);
            spans.push_back(c.t[j]);
            spans.push_back(c.i[j] - ci);
            ct = c.t[j];
            ci = c.i[j];
        }
        counts[p] = static_cast<int32_t>(c.t.size());
    }
    fwrite(counts.data(), sizeof(int32_t), counts.size(), out);
    fwrite(spans.data(), sizeof(int32_t), spans.size(), out);
    return bad;
}

// The general n-order tree (orders 3..5), driven as the kernel drives it: after every word
// the final pending cuts go to the sink in time order (release); they must arrive strictly
// increasing and the tree's ordering flag must stay clear.  The pending-cut ring holds
// `cap` cuts; a pixel that needs more sets the tree's full flag (exit status 4), and the
// largest number of cuts pending at a word end over all pixels goes to stderr.
template <int N, int RL>
int run_tree(const std::vector<uint8_t> &s, int64_t P, int T, int64_t pitch, int cap, FILE *out) {
    std::vector<int32_t> counts(P, 0), spans;
    std::vector<int> pend_t(cap), pend_i(cap);
    int bad = 0, max_np = 0;
    auto *sc = new spk::TreeScan<N, RL>;
    std::vector<int> deep(spk::TreeScan<N, RL>::NF * spk::TreeScan<N, RL>::DEEPN);
    for (int64_t p = 0; p < P; ++p) {
        sc->init(deep.data(), pend_t.data(), pend_i.data(), 1, cap);
        Cuts c;
        int t0 = -1;
        for (int base = 0; base < T; base += 32) {
            uint32_t w = 0;
            for (int k = 0; k < 32 && base + k < T; ++k)
                w |= static_cast<uint32_t>((s[(base + k) * pitch + p / 8] >> (p % 8)) & 1) << k;
            if (sc->last_t < 0 && w) {
                t0 = base + __builtin_ctz(w);
                sc->first_spike(t0);
                w &= w - 1;
            }
            if (w == 0xffffffffu && sc->absorb_ones(base)) w = 0;
            while (w) {
                const int b = __builtin_ctz(w);
                w &= w - 1;
                sc->spike(base + b, c);
            }
            if (sc->np > max_np) max_np = sc->np;
            sc->release(c);
        }
        sc->finish(c);
        if (sc->bad & spk::TREE_BAD_ORDER) bad |= 1;
        if (sc->bad & spk::TREE_BAD_FULL) bad |= 4;
        for (size_t j = 1; j < c.t.size(); ++j)
            if (c.t[j] <= c.t[j - 1]) bad |= 1;
        int ct = t0, ci = -1;
        for (size_t j = 0; j < c.t.size(); ++j) {
            spans.push_back(ct);
            spans.push_back(c.t[j]);
            spans.push_back(c.i[j] - ci);
            ct = c.t[j];
            ci = c.i[j];
        }
        counts[p] = static_cast<int32_t>(c.t.size());
    }
    delete sc;
    fprintf(stderr, "max_pending %d\n", max_np);
    fwrite(counts.data(), sizeof(int32_t), counts.size(), out);
    fwrite(spans.data(), sizeof(int32_t), spans.size(), out);
    return bad;
}

}  // namespace

int main(int argc, char **argv) {
    if (argc != 7 && argc != 8) {
        fprintf(stderr, "usage: scan_host stream.bin P T pitch order[l] out.bin [ring capacity, orders 3..5]\n");
        return 2;
    }
    const int cap = argc == 8 ? atoi(argv[7]) : 1 << 16;
    if (cap < 1 || (cap & (cap - 1))) {
        fprintf(stderr, "the ring capacity must be a power of two\n");
        return 2;
    }
    const int64_t P = atoll(argv[2]), pitch = atoll(argv[4]);
    const int T = atoi(argv[3]), order = atoi(argv[5]);
    const bool reg = strchr(argv[5], 'l') == nullptr;  // "3l": every level's node state indexed by node
    std::vector<uint8_t> s(static_cast<size_t>(pitch) * T);
    FILE *f = fopen(argv[1], "rb");
    if (!f || fread(s.data(), 1, s.size(), f) != s.size()) return 2;
    fclose(f);
    FILE *out = fopen(argv[6], "wb");
    if (!out) return 2;
    if (order < 1 || order > spk::TREE_MAX) return 2;
    const int bad = order == 1   ? run<1>(s, P, T, pitch, out)
                    : order == 2 ? run<2>(s, P, T, pitch, out)
                    : order == 3 ? (reg ? run_tree<3, 3>(s, P, T, pitch, cap, out)
                                        : run_tree<3, 1>(s, P, T, pitch, cap, out))
                    : order == 4 ? (reg ? run_tree<4, 3>(s, P, T, pitch, cap, out)
                                        : run_tree<4, 1>(s, P, T, pitch, cap, out))
                                 : (reg ? run_tree<5, 3>(s, P, T, pitch, cap, out)
                                        : run_tree<5, 1>(s, P, T, pitch, cap, out));
    fclose(out);
    if (bad)
        fprintf(stderr, "property failed: %s%s%s\n", bad & 1 ? "order " : "", bad & 2 ? "frontier " : "",
                bad & 4 ? "tree pending ring full" : "");
    return bad == 4 ? 4 : bad ? 3 : 0;
}
