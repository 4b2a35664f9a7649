// Host-side 1-D rules and rule blocks of libsg (see sg_rules.cpp).
#pragma once
#include "sg_internal.h"

#ifdef __cplusplus
extern "C" {
#endif

// Nodes of the level-`level` rule of `kind` (1 trapezoid, 2 CC, 4 GL); 0 if invalid.
int sg_level_nodes(int kind, int level);

// Level-`level` rule on [0,1], nodes ascending.  Returns the node count.
int sg_rule_level(int kind, int level, double *x, double *w);

// Block of kind `bk` (SG_BLK_*) at excess k >= 1: nodes/weights on [0,1].
// x, w need room for 2 * 4097 entries.  Returns the node count (0 if invalid).
int sg_block(int kind, int bk, int k, double *x, double *w);

// Node count of a block without building it.
int sg_block_size(int kind, int bk, int k);

#ifdef __cplusplus
}
#endif
