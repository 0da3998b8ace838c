// FP64 reduction (PTCA_FP64): NT = 1, 2, 4, 5 -> matrix orders up to 160
// (shared memory limits FP64 to about 144).
#define PTCA_T double
#define PTCA_SYM(x) x##_f64
#define PTCA_NT_LIST(X) X(1) X(2) X(4) X(5)
#include "kernels_prec.inc"
