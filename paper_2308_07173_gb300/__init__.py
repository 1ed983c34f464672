"""GB300-native nearest-points search + neighbourhood covariance.

The data-parallel step of GICP-style LiDAR scan registration (Sec. III-C1,
Eq. 18-20): for every query point, its k nearest neighbours in a
device-resident target map (a voxel-hash grid, Sec. III-C3) and the 3x3
covariance of that neighbourhood, optionally plane-regularised.

* ``pc``        -- ctypes binding of the C ABI in include/pc.h (libpc.so)
* ``workloads`` -- seeded synthetic LiDAR scans and race-track maps
* ``autotune``  -- launch-shape / cell-size tuner with a JSON cache
* ``serve``     -- continuous-batching request loop with p50/p99 latency
"""
__version__ = "0.1.0"
