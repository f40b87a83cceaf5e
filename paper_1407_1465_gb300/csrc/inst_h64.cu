#define RSAGPU_UNIT 64
#include "inst_unit.cuh"
