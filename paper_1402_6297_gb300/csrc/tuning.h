// Written by autotune.py: the complex64 product's kernel schedule for this GPU
// (grid sizes 48,64,96; score = sum of product time per voxel; a change is
// taken only when it gains more than 3%, the run-to-run spread).
#pragma once
#ifndef NFS_N1_32
#define NFS_N1_32 8
#endif
#ifndef NFS_N1_48
#define NFS_N1_48 8
#endif
#ifndef NFS_N1_64
#define NFS_N1_64 8
#endif
#ifndef NFS_N1_96
#define NFS_N1_96 12
#endif
#ifndef NFS_N1_128
#define NFS_N1_128 16
#endif
#ifndef NFS_PLANE_MINB
#define NFS_PLANE_MINB 3
#endif
#ifndef NFS_Z_MINB
#define NFS_Z_MINB 3
#endif
#ifndef NFS_ZTILE_C64
#define NFS_ZTILE_C64 16
#endif
#ifndef NFS_C64_PAIRS
#define NFS_C64_PAIRS 0
#endif
