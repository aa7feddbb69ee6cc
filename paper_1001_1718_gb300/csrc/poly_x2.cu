// Register-window kernels for the asymmetric map at exactly x2 vertically
// (two output rows per source position, aligned staging): the POLY_FIX 2
// set of poly.cu, compiled as its own translation unit.
#define POLY_MODE 1
#define POLY_FIX 2
#include "poly.cu"
