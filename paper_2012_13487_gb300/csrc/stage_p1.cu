// Fused LSRK stage kernel instantiated for polynomial degree 1.
#define FEDBM_P 1
#define FEDBM_STAGE_ENTRY_NAME stage_entry_p1
#include "stage_impl.cuh"
