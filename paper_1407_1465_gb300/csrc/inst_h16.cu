#define RSAGPU_UNIT 16
#include "inst_unit.cuh"
