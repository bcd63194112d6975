// Host-only checks of the workspace layout (no GPU needed): every region
// 256-byte aligned and disjoint from the next, the per-call zeroed range
// covering exactly the control records the kernels expect to be zero, and
// the self-resetting slots outside it.  Prints one line per failure and
// exits non-zero if there is any.
#include <cstdio>
#include <string>
#include <vector>

#include "../paper_2303_10581_gb300/csrc/common.cuh"

using namespace ch;

struct Region {
    const char *name;
    size_t at, bytes;
};

static int fails = 0;
#define CHECK(cond, ...)                 \
    do {                                 \
        if (!(cond)) {                   \
            std::printf(__VA_ARGS__);    \
            std::printf("\n");           \
            ++fails;                     \
        }                                \
    } while (0)

static void check_single(int64_t n, int64_t sets)
{
    const Layout L = make_layout(n, sets);
    const size_t ft = (size_t)L.filt_tiles, st = (size_t)L.sort_tiles, nc = (size_t)L.n_chunks;
    const size_t nn = (size_t)L.n;
    std::vector<Region> r = {
        {"persist", L.persist, sizeof(Persist)},
        {"extctrl", L.extctrl, sizeof(ExtCtrl)},
        {"oct", L.oct, sizeof(Octagon)},
        {"ext8", L.ext8, 32},
        {"kxctrl", L.kxctrl, sizeof(KxCtrl)},
        {"kpoly", L.kpoly, sizeof(KPoly)},
        {"ctrl", L.ctrl, sizeof(Ctrl)},
        {"filt_status", L.filt_status, ft * 8},
        {"kgon_ctrl", L.kgon_ctrl, sizeof(KgonCtrl)},
        {"fan2", L.fan2, sizeof(Fan2Ctrl)},
        {"fan2_slot", L.fan2_slot, (size_t)L.fan2_bins * 8},
        {"node_cnt", L.node_cnt, (size_t)L.n_nodes * 4},
        {"emit_status0", L.emit_status[0], (size_t)L.emit_tiles * 8},
        {"emit_status1", L.emit_status[1], (size_t)L.emit_tiles * 8},
        {"keys0", L.keys[0], nn * 4},
        {"keys1", L.keys[1], nn * 4},
        {"pay0", L.pay[0], nn * 8},
        {"pay1", L.pay[1], nn * 8},
        {"sort_status0", L.sort_status[0], st * 256 * 4},
        {"sort_status1", L.sort_status[1], st * 256 * 4},
        {"chain_pos0", L.chain_pos[0], nc * kChainStride * 4},
        {"chain_pt0", L.chain_pt[0], nc * kChainStride * 8},
        {"chain_pos1", L.chain_pos[1], nc * kChainStride * 4},
        {"chain_pt1", L.chain_pt[1], nc * kChainStride * 8},
        {"chunk", L.chunk, nc * 8 * 4},
        {"node", L.node, (size_t)L.n_nodes * 4 * 4},
        {"emit_off0", L.emit_off[0], (nc + 1) * 4},
        {"emit_off1", L.emit_off[1], (nc + 1) * 4},
        {"keep_bits", L.keep_bits, ft * kFiltThreads * 2},
        {"filt_bsum", L.filt_bsum, (size_t)kFiltMaxBlocks * 4},
        {"kgon", L.kgon, sizeof(Kgon)},
        {"utmp", L.utmp, nn * 4},
        {"spec", L.spec, sizeof(SpecCtrl)},
        {"p0", L.p0, 256},
        {"learn", L.learn, sizeof(LearnScratch)},
        {"fan2_v", L.fan2_v, (size_t)L.fan2_bins * 8},
    };
    for (size_t i = 0; i < r.size(); ++i) {
        CHECK(r[i].at % 256 == 0, "n=%lld sets=%lld: %s not 256-aligned", (long long)n, (long long)sets, r[i].name);
        const size_t end = r[i].at + r[i].bytes;
        const size_t next = i + 1 < r.size() ? r[i + 1].at : L.total;
        CHECK(end <= next, "n=%lld sets=%lld: %s overlaps the next region", (long long)n, (long long)sets, r[i].name);
    }
    // the zeroed range: ctrl .. end of emit_status[1]
    const size_t z0 = L.ctrl, z1 = L.ctrl + L.zero_words * 8;
    for (const char *need : {"ctrl", "filt_status", "kgon_ctrl", "fan2", "fan2_slot", "node_cnt", "emit_status0",
                             "emit_status1"})
        for (const Region &x : r)
            if (std::string(x.name) == need)
                CHECK(x.at >= z0 && x.at + x.bytes <= z1, "n=%lld: %s outside the zeroed range", (long long)n, need);
    for (const char *keep : {"persist", "extctrl", "kxctrl", "keys0"})
        for (const Region &x : r)
            if (std::string(x.name) == keep)
                CHECK(x.at + x.bytes <= z0 || x.at >= z1, "n=%lld: %s inside the zeroed range", (long long)n, keep);
    // the fan's per-tile scratch fits the filter's
    CHECK(ft * kFiltThreads * 2 >= ft * 512, "keep bits per tile");
    // the second fan level: tables for large single sets only; its keep
    // bits, tile counts and block totals reuse the filter's (one survivor
    // tile per point tile at most)
    CHECK(L.fan2_bins == ((sets == 0 && n >= kFan2MinN) ? kFan2Bins : 0), "n=%lld sets=%lld: fan2 tables",
          (long long)n, (long long)sets);
    if (sets > 0) {
        const BatchLayout B = make_batch_layout(L, sets);
        CHECK(B.sets >= L.total && B.sets % 256 == 0, "sets=%lld: batch records overlap", (long long)sets);
        CHECK(B.zero_begin <= B.bctrl && B.hist + (size_t)sets * kSortPasses * 256 * 4 <= B.zero_end,
              "sets=%lld: batch zero range", (long long)sets);
        CHECK(B.sc_off[1] + (size_t)(B.tiles_max + 1) * 4 <= B.total, "sets=%lld: batch total", (long long)sets);
        CHECK(B.lower == L.keys[1], "lower chains alias the second key buffer");
    }
}


int main()
{
    const int64_t sizes[] = {1, 2, 4095, 4096, 4097, 100003, (int64_t)1 << 20, 100000000, (int64_t)1 << 26, 1000000000};
    for (int64_t n : sizes) {
        check_single(n, 0);
        for (int64_t sets : {1, 100, 4096}) check_single(n, sets);
    }
    if (fails) std::printf("%d failures\n", fails);
    else std::printf("layout ok\n");
    return fails ? 1 : 0;
}
