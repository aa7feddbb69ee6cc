// Register-window kernels with shifted staging (source rows at any element
// alignment): the POLY_MODE 2 half of poly.cu, compiled as its own
// translation unit so both halves build in parallel.
#define POLY_MODE 2
#include "poly.cu"
