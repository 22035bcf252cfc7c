// Compile-time checks of the point-group count at the edges of the point
// range the entry points accept (1 .. 2^32 - 1).  Compiling this file is the
// test: a wrong count fails a static_assert.
#include "mmr_points.cuh"

using mmr::groups_of;
using mmr::kBF16;
using mmr::kF16;
using mmr::kF32;

static_assert(groups_of<kF32>(0u) == 0u, "no points, no groups");
static_assert(groups_of<kF32>(1u) == 1u, "one partial group");
static_assert(groups_of<kF32>(4u) == 1u && groups_of<kF32>(5u) == 2u, "4 FP32 points per group");
static_assert(groups_of<kF16>(8u) == 1u && groups_of<kF16>(9u) == 2u, "8 binary16 points per group");
// n + G - 1 would wrap in 32 bits for the largest counts
static_assert(groups_of<kF32>(0xFFFFFFFFu) == 0x40000000u, "2^32 - 1 FP32 points");
static_assert(groups_of<kF32>(0xFFFFFFFDu) == 0x40000000u, "2^32 - 3 FP32 points");
static_assert(groups_of<kF16>(0xFFFFFFFFu) == 0x20000000u, "2^32 - 1 binary16 points");
static_assert(groups_of<kBF16>(0xFFFFFFF9u) == 0x20000000u, "2^32 - 7 bfloat16 points");
static_assert(groups_of<kBF16>(0xFFFFFFF8u) == 0x1FFFFFFFu, "2^32 - 8 bfloat16 points");

int main() { return 0; }
