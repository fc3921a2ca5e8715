"""GB300-native solver for the hot path of the non-gray phonon BTE (arXiv:2305.19400, Sec. 3)."""
