// Sizes shared by the host plan builder and the kernels.
#pragma once

namespace kifmm {

// Number of M2L offsets: {-3..3}^3 minus {-1..1}^3.
constexpr int kNumOffsets = 316;
// Rows (targets) of one M2L tile.
constexpr int kTileRows = 128;
// Finest level representable by the 16-bit integer coordinates.
constexpr int kKeyBits = 16;

} // namespace kifmm
