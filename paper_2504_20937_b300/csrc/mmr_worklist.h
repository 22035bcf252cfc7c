// The batch frame's work list (plain C++, no CUDA): the order in which the
// persistent CTAs of one frame take their items.
//
// A point item is up to `chunk_groups` point groups of one cloud, a pixel
// item up to `chunk_quads` quads of one cloud's framebuffer (every cloud has
// at least one: it owns the ragged tail of pixels).  Every cloud's point items
// come in cloud order; a cloud's pixel items follow once `lag` further point
// items have been listed, or at the end.  A cloud's pixel items therefore
// always come after all of its point items, which is what lets a pixel item
// wait for its cloud's point items without ever waiting on an item that has
// not been handed out.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

namespace mmr {

// Item word x: the cloud, with this bit set for a pixel item; y: the first
// point group (point item) or quad (pixel item).
constexpr uint32_t kPixelItem = 0x80000000u;

struct WorkItem {
    uint32_t x, y;
};

// groups[c] / quads[c]: point groups and whole quads of cloud c.  Fills
// point_items[c] with the number of point items of cloud c.
inline std::vector<WorkItem> build_work_list(const std::vector<uint32_t> &groups, const std::vector<uint32_t> &quads,
                                             uint32_t chunk_groups, uint32_t chunk_quads, uint64_t lag,
                                             std::vector<uint32_t> &point_items)
{
    const size_t count = groups.size();
    std::vector<WorkItem> items;
    point_items.assign(count, 0);
    std::vector<std::pair<uint32_t, uint64_t>> done;   // (cloud, point items listed after its last one)
    uint64_t listed = 0;
    size_t head = 0;
    auto push_pixels = [&](uint32_t c) {
        uint32_t q = 0;
        do {
            items.push_back(WorkItem{c | kPixelItem, q});
            q += chunk_quads;
        } while (q < quads[c]);
    };
    for (uint32_t c = 0; c < (uint32_t)count; ++c) {
        for (uint32_t g = 0; g < groups[c]; g += chunk_groups) {
            items.push_back(WorkItem{c, g});
            point_items[c] += 1;
            ++listed;
            while (head < done.size() && listed - done[head].second >= lag)
                push_pixels(done[head++].first);
        }
        done.push_back({c, listed});
    }
    while (head < done.size())
        push_pixels(done[head++].first);
    return items;
}

}  // namespace mmr
