"""B300-native (sm_103a) real-time 3D reconstruction from single-photon lidar
histograms: the C-ABI CUDA library (csrc/, built to lib/librt3d.so) and its
thin Python binding (rt3d.py).  Importing the package loads nothing; the
library is loaded on first use and its absence is an error."""
