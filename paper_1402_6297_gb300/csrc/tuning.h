// Written by autotune.py: the complex64 product's kernel schedule for this GPU
// (grid sizes 48,64,96; score = sum of product time per voxel).
#pragma once
#define NFS_N1_32 8
#define NFS_N1_48 8
#define NFS_N1_64 8
#define NFS_N1_96 8
#define NFS_N1_128 16
#define NFS_PLANE_MINB 3
#define NFS_Z_MINB 3
#define NFS_ZTILE_C64 16
#define NFS_C64_PAIRS 0
