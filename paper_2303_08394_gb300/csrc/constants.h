// Sizes shared by the host plan builder and the kernels.
#pragma once

namespace kifmm {

// Number of M2L offsets: {-3..3}^3 minus {-1..1}^3.
constexpr int kNumOffsets = 316;
// Rows (targets) of one M2L tile.
constexpr int kTileRows = 128;
// Finest level representable by the 16-bit integer coordinates.
constexpr int kKeyBits = 16;
// Width groups of the leaf pass: leaves of up to 16 T points take T targets
// per lane, T = 1 .. kLeafWidths (larger leaves join the widest group).
constexpr int kLeafWidths = 8;

} // namespace kifmm
