// Tile geometry shared by the host planner and the device kernels.
#pragma once

namespace am {
constexpr int TILE = 32;            // edge of the dense tiles of the local factor storage
constexpr int TILE2 = TILE * TILE;
}  // namespace am
