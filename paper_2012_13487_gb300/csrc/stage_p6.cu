// Fused LSRK stage kernel instantiated for polynomial degree 6.
#define FEDBM_P 6
#define FEDBM_STAGE_ENTRY_NAME stage_entry_p6
#include "stage_impl.cuh"
