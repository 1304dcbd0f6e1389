"""GB300-native SAQ encoder (arXiv 2509.12086): Python binding package."""
