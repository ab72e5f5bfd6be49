"""BDL-tree (arXiv 2112.06188) hot path for GB300 (sm_103a)."""
