"""GB300-native (sm_103a) implementation of the data-parallel hot path of "CUDA-Accelerated Soft
Robot Neural Evolution with Large Language Model Supervision" (arXiv 2405.00698).

    build        -- in-tree nvcc build of libvoxsim.so
    voxsim       -- ctypes binding of the C ABI (include/voxsim.h)
    workloads    -- seeded synthetic populations and parameter presets
"""
