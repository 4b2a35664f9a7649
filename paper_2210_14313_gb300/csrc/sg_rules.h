// Host-side 1-D rules and rule blocks of libsg (see sg_rules.cpp).
#pragma once
#include "sg_internal.h"

// Rule kinds 1 trapezoid, 2 Clenshaw-Curtis, 3 Gauss-Patterson, 4 Gauss-Legendre,
// with SG_KIND_SLOW OR'ed in for the accuracy-level growth of Section 5.4
// (level l uses the smallest member exact to degree 2l - 1).
#define SG_KIND_SLOW 16
#define SG_GP_MEMBERS 6  // Gauss-Patterson members of 1 .. 63 nodes

#ifdef __cplusplus
extern "C" {
#endif

// Member (1-based) of the rule family that level `level` uses; 0 if invalid.
int sg_level_member(int kind, int level);

// Nodes of the level-`level` rule of `kind`; 0 if invalid.
int sg_level_nodes(int kind, int level);

// Level-`level` rule on [0,1], nodes ascending.  Returns the node count.
int sg_rule_level(int kind, int level, double *x, double *w);

// Block of kind `bk` (SG_BLK_*) at excess k >= 1: nodes/weights on [0,1]
// (SG_BLK_NEW: the nodes level k+1 adds, weight 1).
// x, w need room for 2 * 4097 entries.  Returns the node count (0 if invalid,
// and for a difference block whose two levels use the same member).
int sg_block(int kind, int bk, int k, double *x, double *w);

// Node count of a block without building it.
int sg_block_size(int kind, int bk, int k);

#ifdef __cplusplus
}
#endif
