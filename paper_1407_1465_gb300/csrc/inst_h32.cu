#define RSAGPU_UNIT 32
#include "inst_unit.cuh"
