// Host-side check of the shared-memory layout of the tensor-memory moving-source kernel:
// this file includes the kernel's translation unit, so it sees the same constants, the
// program struct and the launcher's size function, and replays on the CPU the offsets the
// kernel derives from them.  Nothing here runs on a GPU.
//
// Checked for every stage count the launcher may pick: the source windows start on 1024-byte
// boundaries (the 128-byte TMA swizzle), the table blocks on 16-byte boundaries (bulk copies),
// the mbarriers on 8-byte boundaries, every tap program's weight rows on 16-byte boundaries
// (16-byte zeroing stores), the fold accumulators on 8-byte boundaries, the regions do not
// overlap and the total fits one CTA's 227 KB; and the stage count the launcher's search picks
// for the tap counts the kernel accepts.
#include "../paper_1502_03162_gb300/csrc/moving_tmem.cu"

#include <cstdio>

namespace {

int failures = 0;

void expect(bool ok, const char *what, int stages, long long value)
{
    if (!ok) {
        std::printf("FAIL %s (stages=%d value=%lld)\n", what, stages, value);
        ++failures;
    }
}

}  // namespace

int main()
{
    using namespace hrir;
    expect(sizeof(Prog) == (size_t)kProgBytes, "program slot = program struct", 0, (long long)sizeof(Prog));
    for (int stages = 2; stages <= kMixMaxStages; ++stages) {
        int ro = -1, po = -1;
        const size_t total = moving_tmem_smem_bytes(stages, kMvMaxK, &ro, &po);
        if (total == 0) continue;   // this stage count does not fit
        const size_t tbls = (size_t)stages * kWinBytes;
        const size_t bars = tbls + (size_t)stages * kStageTableBytes;
        const size_t bars_end = bars + (size_t)(2 * stages + 4 * NQ) * 8 + 16 + kMixMaxStages * 4;
        for (int s = 0; s < stages; ++s) {
            expect((s * (size_t)kWinBytes) % 1024 == 0, "window 1024-byte aligned", stages, s);
            expect((tbls + s * (size_t)kStageTableBytes) % 16 == 0, "table block 16-byte aligned", stages, s);
        }
        expect(bars % 8 == 0, "mbarriers 8-byte aligned", stages, (long long)bars);
        expect((size_t)po >= bars_end, "programs after the barriers", stages, po);
        for (int i = 0; i < 2 * NQ * 2; ++i) {
            const size_t prog = (size_t)po + (size_t)i * sizeof(Prog);
            expect((prog + offsetof(Prog, w)) % 16 == 0, "program weights 16-byte aligned", stages, i);
            expect((prog + offsetof(Prog, col)) % 4 == 0, "program columns 4-byte aligned", stages, i);
        }
        expect((size_t)po + (size_t)kProgsBytes <= (size_t)ro, "programs before the accumulators", stages, ro);
        expect(ro % 8 == 0, "fold accumulators 8-byte aligned", stages, ro);
        expect((size_t)ro + (size_t)kRunAccBytes == total, "accumulators end the layout", stages, (long long)total);
        expect(total <= 227 * 1024, "fits one CTA", stages, (long long)total);
    }
    // the launcher's search (deepest ring that fits) for every tap count the kernel takes
    for (int k = 4; k <= kMvMaxK; k += 4) {
        int stages = kMixMaxStages;
        for (; stages >= 2; --stages)
            if (moving_tmem_smem_bytes(stages, k, nullptr, nullptr) != 0) break;
        expect(stages >= 5, "at least 5 stages", stages, k);
    }
    if (failures == 0) std::printf("ok\n");
    return failures == 0 ? 0 : 1;
}
