// Fused LSRK stage kernel instantiated for polynomial degree 5.
#define FEDBM_P 5
#define FEDBM_STAGE_ENTRY_NAME stage_entry_p5
#include "stage_impl.cuh"
