// FP32 reduction (PTCA_MIXED) in one-warp CTAs -- one warp per matrix -- for
// matrix orders up to 32 (2x2x... windows of at most 16 sites: the Hubbard
// 4x4 and Holstein chain clusters): every vector entry still has its own
// thread, barriers are warp-wide, and many matrices are resident per SM.
// Sweep kernels only.
#define PTCA_T float
#define PTCA_SYM(x) x##_f32w1
#define PTCA_NT_LIST(X) X(1)
#define PTCA_NWP 1
#define PTCA_AUX 0
#include "kernels_prec.inc"
