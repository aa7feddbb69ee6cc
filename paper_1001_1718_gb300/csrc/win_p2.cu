// Register-window forward kernels, part 2 of win.cu (see its header).
#define WIN_PART 2
#include "win.cu"
