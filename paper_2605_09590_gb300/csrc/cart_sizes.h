// Supported transform lengths and their two-factor splits N = N1 * N2.
// X(N, N1, N2): N1 values per "frequency job", N2 per "row job".
#pragma once
#define PICO_SIZES_A(X) \
  X(32, 8, 4) X(40, 10, 4) X(48, 12, 4) X(64, 8, 8) X(80, 10, 8) X(96, 12, 8) X(120, 15, 8) X(128, 16, 8)
#define PICO_SIZES_B(X) \
  X(160, 20, 8) X(192, 12, 16) X(240, 15, 16) X(256, 16, 16) X(320, 20, 16) X(384, 24, 16)
#define PICO_SIZES(X) PICO_SIZES_A(X) PICO_SIZES_B(X)
