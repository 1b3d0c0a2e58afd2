// Translation units of the element-operator instantiations.  Each entry
// X(name, law, dim, lobatto_mask, gauss_mask) becomes one compilation of
// ops_inst.cu (bit P of a mask = P nodes per direction compiled).  The build
// script reads this list, so it is the single place that decides what exists.
#pragma once
#define HBPC_OPS_UNITS(X)            \
  X(adv1, 0, 1, 0x1FC, 0x18)         \
  X(adv2, 0, 2, 0x1FC, 0x18)         \
  X(adv3, 0, 3, 0x1FC, 0x0)          \
  X(bur1, 1, 1, 0x1F8, 0x18)         \
  X(bur2, 1, 2, 0x1F8, 0x18)         \
  X(bur3, 1, 3, 0x78, 0x0)           \
  X(eul1, 2, 1, 0x78, 0x18)          \
  X(eul2a, 2, 2, 0x18, 0x18)         \
  X(eul2b, 2, 2, 0x60, 0x0)          \
  X(eul3a, 2, 3, 0x18, 0x0)          \
  X(eul3b, 2, 3, 0x60, 0x0)          \
  X(ns2a, 3, 2, 0x18, 0x18)          \
  X(ns2b, 3, 2, 0x60, 0x0)           \
  X(ns3a, 3, 3, 0x18, 0x0)           \
  X(ns3b, 3, 3, 0x40, 0x0)           \
  X(ns3c, 3, 3, 0x20, 0x0)
