"""GB300-native ADAGIO: data-aware near-isometric linear embedding with an exhaustive distortion certificate."""
