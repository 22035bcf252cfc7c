// Checks the batch frame's work list (paper_2504_20937_b300/csrc/mmr_worklist.h)
// on random batches: every point and pixel item exactly once, point items in
// cloud order, every cloud's pixel items after all of its point items (what
// makes a pixel item's wait end), and at least `lag` point items between a
// cloud's last point item and its first pixel item unless the list runs out
// of point items first.  Prints "ok <cases>" or the first failure.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "mmr_worklist.h"

static int fail(const char *what, int trial)
{
    std::printf("FAIL trial %d: %s\n", trial, what);
    return 1;
}

int main()
{
    std::mt19937_64 rng(20250503);
    int cases = 0;
    for (int trial = 0; trial < 3000; ++trial) {
        const int count = 1 + (int)(rng() % (trial < 100 ? 4 : 300));
        std::vector<uint32_t> groups(count), quads(count);
        for (int c = 0; c < count; ++c) {
            groups[c] = 1 + (uint32_t)(rng() % (rng() % 4 == 0 ? 20000 : 200));
            quads[c] = (uint32_t)(rng() % (rng() % 4 == 0 ? 300000 : 3000));   // 0: a cloud of 1..3 pixels
        }
        const uint32_t chunk_groups = 1 + (uint32_t)(rng() % 4096);
        const uint32_t chunk_quads = 4 * chunk_groups;
        const uint64_t lag = rng() % 3 == 0 ? 0 : (rng() % 5000);
        std::vector<uint32_t> per_cloud;
        const std::vector<mmr::WorkItem> items =
            mmr::build_work_list(groups, quads, chunk_groups, chunk_quads, lag, per_cloud);
        std::vector<uint32_t> next_group(count, 0), next_quad(count, 0), pixels_seen(count, 0);
        std::vector<int64_t> last_point(count, -1), first_pixel(count, -1);
        std::vector<uint64_t> points_before(items.size() + 1, 0);   // point items among items[0..k)
        int prev_cloud = 0;
        for (size_t k = 0; k < items.size(); ++k) {
            const mmr::WorkItem w = items[k];
            const uint32_t c = w.x & ~mmr::kPixelItem;
            points_before[k + 1] = points_before[k] + ((w.x & mmr::kPixelItem) ? 0 : 1);
            if (c >= (uint32_t)count)
                return fail("cloud out of range", trial);
            if (w.x & mmr::kPixelItem) {
                if (w.y != next_quad[c])
                    return fail("pixel items of a cloud missing, repeated or out of order", trial);
                next_quad[c] += chunk_quads;
                pixels_seen[c] += 1;
                if (first_pixel[c] < 0)
                    first_pixel[c] = (int64_t)k;
                if (last_point[c] < 0 || next_group[c] < groups[c])
                    return fail("a pixel item before all of its cloud's point items", trial);
            } else {
                if ((int)c < prev_cloud)
                    return fail("point items not in cloud order", trial);
                prev_cloud = (int)c;
                if (w.y != next_group[c])
                    return fail("point items of a cloud missing, repeated or out of order", trial);
                next_group[c] += chunk_groups;
                last_point[c] = (int64_t)k;
            }
        }
        const uint64_t total_points = points_before[items.size()];
        for (int c = 0; c < count; ++c) {
            if (next_group[c] < groups[c])
                return fail("point groups not covered", trial);
            if (per_cloud[c] != (groups[c] + chunk_groups - 1) / chunk_groups)
                return fail("per-cloud point item count", trial);
            if (pixels_seen[c] == 0 || next_quad[c] < quads[c] || (quads[c] > 0 && next_quad[c] - chunk_quads >= quads[c]))
                return fail("pixel quads not covered exactly", trial);
            const uint64_t between = points_before[first_pixel[c]] - points_before[last_point[c] + 1];
            const uint64_t after = total_points - points_before[last_point[c] + 1];
            if (between < (lag < after ? lag : after))
                return fail("fewer than `lag` point items between a cloud's points and its pixels", trial);
        }
        ++cases;
    }
    std::printf("ok %d\n", cases);
    return 0;
}
