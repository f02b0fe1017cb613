"""GB300-native k x k median filter by hierarchical tiling (arXiv 2507.19926)."""
