"""CPU oracle (test infrastructure only): plain FP64 reference of the octree-block multigrid method."""
