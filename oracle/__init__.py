"""FP64 CPU oracle of the voxel soft-robot hot path (test infrastructure only)."""
