// Exact-decision descent kernels (KRP_PREC_EXACT, R <= 32): the descent of
// descent_fast.cu compiled with its exact-decision code, in a translation unit
// of its own.
#define KRP_DESCENT_EXACT_TU 1
#include "descent_fast.cu"
