"""GB300-native matrix-free ghost-penalty operator (y = G x) for Cartesian CutFEM meshes."""
