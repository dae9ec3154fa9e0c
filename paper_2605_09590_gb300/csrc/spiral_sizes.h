// Grid lengths of the Toeplitz / 2-D passes and their splits L = P1 * P2
// (X(L, P1, P2)).  Spiral operators use L = 2N; 2-D Cartesian masks L = N.
#pragma once
#define PICO_GRID_SIZES_A(X) X(64, 8, 8) X(80, 10, 8) X(96, 12, 8) X(128, 16, 8) X(160, 20, 8) X(192, 12, 16)
#define PICO_GRID_SIZES_B(X) X(240, 15, 16) X(256, 16, 16) X(320, 20, 16) X(384, 24, 16) X(480, 30, 16)
#define PICO_GRID_SIZES(X) PICO_GRID_SIZES_A(X) PICO_GRID_SIZES_B(X)
