#define RSAGPU_UNIT 48
#include "inst_unit.cuh"
