// Fused LSRK stage kernel instantiated for polynomial degree 2.
#define FEDBM_P 2
#define FEDBM_STAGE_ENTRY_NAME stage_entry_p2
#include "stage_impl.cuh"
