// Grid lengths L = 2N of the spiral (Toeplitz / gridding) kernels and their
// splits L = P1 * P2 (X(L, P1, P2)).
#pragma once
#define PICO_GRID_SIZES(X) \
  X(128, 16, 8) X(160, 20, 8) X(192, 12, 16) X(240, 15, 16) X(320, 20, 16) X(384, 24, 16) X(480, 30, 16)
