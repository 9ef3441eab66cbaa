"""GB300-native long-range molecular dynamics (HMF, Ring, 2D self-gravitating)."""
